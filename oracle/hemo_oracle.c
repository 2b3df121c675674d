/*
 * CPU oracle for the coupled lattice-Boltzmann / immersed-boundary time step
 * of the HemoCell method (Zavodszky et al., "Cellular blood flow modelling
 * with HemoCell").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg load this library; the product
 * (the CUDA library) never calls it and shares no code with it.
 *
 * Plain FP64 loops, two population arrays and pull streaming, in the order
 * the method states.  The loops over independent nodes, cells and vertices
 * carry OpenMP annotations (threads set by ora_set_threads, 1 by default);
 * each iteration writes only its own node, cell or vertex, so the results
 * do not depend on the thread count.  The spreading loop, which sums into
 * shared nodes, stays serial.  Paper passages followed:
 *   Sec. 2.2  BGK lattice-Boltzmann update (eq. for f_i(x+e_i, t+1)), the
 *             moments rho = sum_i f_i and u = sum_i f_i e_i / rho, the
 *             second-order equilibrium w_i rho [1 + 3 e.u + 9/2 (e.u)^2 -
 *             3/2 u^2], nu = c_s^2 (tau - 1/2), c_s = 1/sqrt(3), D3Q19.
 *   Sec. 2.3  explicit immersed-boundary coupling through external force
 *             terms: lattice velocity interpolated to the membrane vertices,
 *             vertex forces spread back onto the lattice;
 *             F_total = F_link + F_bend + F_area + F_volume.
 *   Sec. 2.5  no-slip walls, periodic boundaries, walls moving in opposite
 *             directions (shear).
 *   Sec. 2.6  vertex positions integrated by Euler or by Adams-Bashforth;
 *             the membrane (constitutive) model may be evaluated less often
 *             than the fluid is updated (time-scale separation).
 * Readings where the paper is silent (each also applied by the CUDA path,
 * which implements them independently):
 *   - forcing: Guo-Zheng-Shi source term with the half-force velocity;
 *   - walls: halfway bounce-back; moving wall adds -6 w_i rho (e_i . u_w)
 *     with rho the density of the colliding fluid node; nodes outside a
 *     non-periodic axis behave as resting walls;
 *   - coupling kernel: Peskin's 4-point kernel (not the 2-point "linear"
 *     kernel), interpolating the post-streaming velocity that includes F/2;
 *     spreading onto wall nodes is discarded; interpolation sees the wall
 *     velocity at wall nodes;
 *   - link: strain-stiffening energy K L0 [eps^2/2 - 1/2 ln(1 - eps^2/m^2)],
 *     K = k_link kBT / p, eps = (L - L0)/L0, m = maximum strain;
 *   - bending: 1/2 k_bend kBT (theta - theta0)^2 per edge, theta the signed
 *     angle between the outward normals of the two triangles of the edge;
 *   - time-scale separation (Sec. 2.6, constant separation N): membrane
 *     forces are evaluated on the steps n = n0, n0 + N, n0 + 2N, ... (n0 the
 *     step at which the setting was made) and held unchanged on the steps in
 *     between; spreading, the fluid update, interpolation and the vertex move
 *     run every step.  The default is N = 1 with Euler;
 *   - adaptive separation (Sec. 2.6 allows an adaptive one; its criterion
 *     is in a cited work that is not available): forces are evaluated on the
 *     first step after the setting and then whenever, at the start of a step,
 *     the largest vertex displacement since the last evaluation exceeds a
 *     tolerance delta, or N steps have passed since it;
 *   - Adams-Bashforth (Sec. 2.6): the two-step explicit form
 *     X^{n+1} = X^n + 3/2 U^n - 1/2 U^{n-1} with dt = 1, U^n the velocity
 *     interpolated at X^n; the first step after the setting is made (no
 *     U^{n-1} yet) is an Euler step;
 *   - nonlinear bending and local area (Sec. 2.3: large deformations give a
 *     highly non-linear response of membrane and cytoskeleton; both terms are
 *     off unless their parameter is set): with a maximum bending deviation
 *     theta_m > 0 the bending energy per edge is k_bend kBT theta_m^2 *
 *     (-1/2) ln(1 - (theta - theta0)^2 / theta_m^2), which is the harmonic
 *     1/2 k_bend kBT (theta - theta0)^2 for small deviations and stiffens
 *     without bound as |theta - theta0| approaches theta_m; with k_local > 0
 *     each triangle adds 1/2 k_local (A_t - A_t0)^2 / A_t0 (A_t0 its rest
 *     area; lattice energy per lattice area);
 *   - internal viscosity (Sec. 1: the cytosol is five times as viscous as the
 *     plasma; Sec. 3: the RBC model has an internal viscosity ratio): with a
 *     ratio lambda != 1, nodes inside a cell membrane at X^n relax with tau_in
 *     = 1/2 + lambda (tau - 1/2) (nu_in = lambda nu).  A node is inside when
 *     the upward ray from it crosses the cell's surface with a net signed
 *     count (sign of the outward normal's z component) of one; a node whose
 *     column passes exactly through a projected triangle edge belongs to the
 *     triangle for which the edge, traversed counter-clockwise as seen from
 *     +z, points in -y, or in +x when horizontal (each shared edge is
 *     evaluated in one canonical vertex order, so its two triangles agree);
 *     a crossing at exactly the node's height counts as below it;
 *   - Lees-Edwards boundary (Sec. 2.5: periodic in every direction with
 *     opposing velocities imposed on two parallel boundaries, cells crossing
 *     it are moved to the other side): along z, the periodic image above the
 *     box is displaced by +D_n in x and moves with +U x^ (the image below by
 *     -D_n, -U), D_n = U n mod nx at step n.  A population streaming across
 *     the plane comes from the image: its value is the linear interpolation
 *     in x, at the displaced position, of the post-collision values of the
 *     two bracketing nodes of the opposite plane, each Galilean-shifted by
 *     f_eq(rho*, u* +/- U) - f_eq(rho*, u*) (rho*, u* the moments of that
 *     node's post-collision populations).  Interpolation and spreading treat
 *     each z-layer of the 4x4x4 stencil that falls in an image with the
 *     vertex's position displaced by -/+D_n in x (and, for interpolation,
 *     the image's velocity +/-U x^).  At the start of a step a cell whose
 *     centroid lies above the box (z >= nz) moves by (-D_n, 0, -nz), below it
 *     by (+D_n, 0, +nz).  Requires a fully periodic lattice without walls;
 *   - area / volume: per cell, in strain form 1/2 k_area ((A - A0)/A0)^2 and
 *     1/2 k_volume ((V - V0)/V0)^2 with k in lattice energy units.  (The form
 *     1/2 k (V - V0)^2 / V0 with k_volume = 20 makes the explicit coupling
 *     diverge within 20 steps on a single red cell in shear; Sec. 2.3 says
 *     the free parameters are tuned for numerical stability.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* ------------------------------------------------------------------------ */
/* D3Q19 velocity set: every c in {-1,0,1}^3 with |c|^2 <= 2, enumerated with */
/* cx slowest and cz fastest; weights 1/3 (|c|^2 = 0), 1/18 (1), 1/36 (2).   */
/* ------------------------------------------------------------------------ */
static int C[Q][3];
static double W[Q];
static int OPP[Q];
static int tables_ready = 0;

static void build_tables(void) {
    if (tables_ready) return;
    int q = 0;
    for (int cx = -1; cx <= 1; ++cx)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cz = -1; cz <= 1; ++cz) {
                int n2 = cx * cx + cy * cy + cz * cz;
                if (n2 > 2) continue;
                C[q][0] = cx; C[q][1] = cy; C[q][2] = cz;
                W[q] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                ++q;
            }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j)
            if (C[j][0] == -C[i][0] && C[j][1] == -C[i][1] && C[j][2] == -C[i][2]) OPP[i] = j;
    tables_ready = 1;
}

void ora_d3q19(int *c, double *w, int *opp) {
    build_tables();
    for (int i = 0; i < Q; ++i) {
        for (int d = 0; d < 3; ++d) c[3 * i + d] = C[i][d];
        w[i] = W[i];
        opp[i] = OPP[i];
    }
}

/* Sec. 2.2 equilibrium */
void ora_equilibrium(double rho, const double *u, double *feq) {
    build_tables();
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        feq[i] = W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Reference of the 16-bit storage form for a row whose reference velocity
 * is (U, 0, 0): for the directions with c_x != 0 the equilibrium deviation
 * f_i^eq(1, (U, 0, 0)) - w_i, zero for the others (the storage form keeps
 * f_i - w_i - K_i in 2 bytes; the oracle computes in FP64 and uses this only
 * to state what the stored values are). */
void ora_storage_reference(double U, double *K) {
    build_tables();
    const double u[3] = {U, 0.0, 0.0};
    double feq[Q];
    ora_equilibrium(1.0, u, feq);
    for (int i = 0; i < Q; ++i) K[i] = C[i][0] != 0 ? feq[i] - W[i] : 0.0;
}

/* Peskin's 4-point kernel (Peskin 2002), piecewise definition */
double ora_phi(double r) {
    double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------------ */
/* membrane mesh type                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nv, nt, ne;
    int *tri;       /* nt*3, outward counter-clockwise */
    int *edge;      /* ne*4: v0, v1, a, b; triangle (v0,v1,a) and (v1,v0,b) */
    double *L0;     /* rest length per edge */
    double *th0;    /* rest dihedral angle per edge */
    double *At0;    /* rest area per triangle */
    double A0, V0;
    double k_link, k_bend, k_area, k_volume, kbt, persistence, max_strain;
    double k_local, theta_m; /* local area modulus; maximum bending deviation (0: harmonic) */
} omesh;

/* Edge table: triangles in order, their directed edges (t0,t1), (t1,t2),
 * (t2,t0); an undirected edge met for the first time gets the next id with
 * v0, v1 in the direction met and a = the triangle's third vertex; the second
 * time (necessarily in the reverse direction for an oriented closed mesh) b
 * = that triangle's third vertex.  Returns the number of edges, or -1 if the
 * mesh is not a consistently oriented closed 2-manifold. */
int ora_build_edges(int nv, int nt, const int *tri, int *edge_out /* capacity 3*nt/2*4 */) {
    int maxe = 3 * nt / 2 + 1;
    int *head = (int *)malloc(sizeof(int) * nv);
    int *next = (int *)malloc(sizeof(int) * maxe);
    int *seen = (int *)malloc(sizeof(int) * maxe); /* times seen */
    for (int v = 0; v < nv; ++v) head[v] = -1;
    int ne = 0, bad = 0;
    for (int t = 0; t < nt && !bad; ++t) {
        for (int k = 0; k < 3; ++k) {
            int a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3], o = tri[3 * t + (k + 2) % 3];
            int lo = a < b ? a : b, hi = a < b ? b : a;
            int found = -1;
            for (int e = head[lo]; e >= 0; e = next[e]) {
                int e0 = edge_out[4 * e], e1 = edge_out[4 * e + 1];
                int elo = e0 < e1 ? e0 : e1, ehi = e0 < e1 ? e1 : e0;
                if (elo == lo && ehi == hi) { found = e; break; }
            }
            if (found < 0) {
                if (ne >= maxe) { bad = 1; break; }
                edge_out[4 * ne + 0] = a;
                edge_out[4 * ne + 1] = b;
                edge_out[4 * ne + 2] = o;
                edge_out[4 * ne + 3] = -1;
                seen[ne] = 1;
                next[ne] = head[lo];
                head[lo] = ne;
                ++ne;
            } else {
                if (seen[found] != 1 || edge_out[4 * found] != b || edge_out[4 * found + 1] != a) { bad = 1; break; }
                edge_out[4 * found + 3] = o;
                seen[found] = 2;
            }
        }
    }
    for (int e = 0; e < ne && !bad; ++e) if (seen[e] != 2) bad = 1;
    free(head); free(next); free(seen);
    return bad ? -1 : ne;
}

/* signed dihedral angle of edge (p0,p1) with wings pa (triangle p0,p1,pa) and
 * pb (triangle p1,p0,pb): atan2(e^ . (n1 x n2), n1 . n2) */
static double dihedral(const double *p0, const double *p1, const double *pa, const double *pb) {
    double e[3], da[3], db[3], n1[3], n2[3], c[3];
    sub3(p1, p0, e); sub3(pa, p0, da); sub3(pb, p0, db);
    cross3(e, da, n1);
    cross3(db, e, n2);
    cross3(n1, n2, c);
    double L = sqrt(dot3(e, e));
    return atan2(dot3(c, e) / L, dot3(n1, n2));
}

static void cell_area_volume(const omesh *m, const double *X, double *A, double *V) {
    double ctr[3] = {0, 0, 0};
    for (int v = 0; v < m->nv; ++v) for (int d = 0; d < 3; ++d) ctr[d] += X[3 * v + d];
    for (int d = 0; d < 3; ++d) ctr[d] /= m->nv;
    double a = 0, vol = 0;
    for (int t = 0; t < m->nt; ++t) {
        const double *x0 = X + 3 * m->tri[3 * t], *x1 = X + 3 * m->tri[3 * t + 1], *x2 = X + 3 * m->tri[3 * t + 2];
        double e1[3], e2[3], n[3], r0[3], r1[3], r2[3], rc[3];
        sub3(x1, x0, e1); sub3(x2, x0, e2); cross3(e1, e2, n);
        a += 0.5 * sqrt(dot3(n, n));
        sub3(x0, ctr, r0); sub3(x1, ctr, r1); sub3(x2, ctr, r2);
        cross3(r1, r2, rc);
        vol += dot3(r0, rc) / 6.0;
    }
    *A = a; *V = vol;
}

static int mesh_init(omesh *m, int nv, int nt, const int *tri, const double *rest, const double *params) {
    m->nv = nv; m->nt = nt;
    m->tri = (int *)malloc(sizeof(int) * 3 * nt);
    memcpy(m->tri, tri, sizeof(int) * 3 * nt);
    m->edge = (int *)malloc(sizeof(int) * 4 * (3 * nt / 2 + 1));
    m->ne = ora_build_edges(nv, nt, tri, m->edge);
    if (m->ne < 0) return -1;
    m->L0 = (double *)malloc(sizeof(double) * m->ne);
    m->th0 = (double *)malloc(sizeof(double) * m->ne);
    for (int e = 0; e < m->ne; ++e) {
        const int *E = m->edge + 4 * e;
        double d[3];
        sub3(rest + 3 * E[1], rest + 3 * E[0], d);
        m->L0[e] = sqrt(dot3(d, d));
        m->th0[e] = dihedral(rest + 3 * E[0], rest + 3 * E[1], rest + 3 * E[2], rest + 3 * E[3]);
    }
    cell_area_volume(m, rest, &m->A0, &m->V0);
    m->At0 = (double *)malloc(sizeof(double) * nt);
    for (int t = 0; t < nt; ++t) {
        double e1[3], e2[3], n[3];
        sub3(rest + 3 * tri[3 * t + 1], rest + 3 * tri[3 * t], e1);
        sub3(rest + 3 * tri[3 * t + 2], rest + 3 * tri[3 * t], e2);
        cross3(e1, e2, n);
        m->At0[t] = 0.5 * sqrt(dot3(n, n));
    }
    m->k_link = params[0]; m->k_bend = params[1]; m->k_area = params[2]; m->k_volume = params[3];
    m->kbt = params[4]; m->persistence = params[5]; m->max_strain = params[6];
    m->k_local = params[7]; m->theta_m = params[8];
    return 0;
}

static void mesh_free(omesh *m) {
    free(m->tri); free(m->edge); free(m->L0); free(m->th0); free(m->At0);
}

/* Sec. 2.3: F_v = -dE/dX_v with E = E_link + E_bend + E_area + E_volume.
 * Adds forces into F (nv*3); returns the four energies in E4 (may be NULL;
 * the local area energy is counted with the area term); writes the cell's
 * area and volume. */
static void membrane_forces(const omesh *m, const double *X, double *F, double *E4, double *Aout, double *Vout) {
    double El = 0, Eb = 0, Ea = 0, Ev = 0;
    /* link: per edge */
    double K = m->k_link * m->kbt / m->persistence;
    double mm = m->max_strain * m->max_strain;
    for (int e = 0; e < m->ne; ++e) {
        const int *E = m->edge + 4 * e;
        double d[3];
        sub3(X + 3 * E[1], X + 3 * E[0], d);
        double L = sqrt(dot3(d, d));
        double eps = (L - m->L0[e]) / m->L0[e];
        El += K * m->L0[e] * (0.5 * eps * eps - 0.5 * log(1.0 - eps * eps / mm));
        double dEdL = K * (eps + eps / (mm - eps * eps));
        for (int k = 0; k < 3; ++k) {
            F[3 * E[0] + k] += dEdL * d[k] / L;
            F[3 * E[1] + k] -= dEdL * d[k] / L;
        }
    }
    /* bending: per edge, gradient of the dihedral angle */
    double kb = m->k_bend * m->kbt;
    for (int e = 0; e < m->ne; ++e) {
        const int *E = m->edge + 4 * e;
        const double *p0 = X + 3 * E[0], *p1 = X + 3 * E[1], *pa = X + 3 * E[2], *pb = X + 3 * E[3];
        double th = dihedral(p0, p1, pa, pb);
        double dth = th - m->th0[e];
        double c;  /* dE/dtheta */
        if (m->theta_m > 0) {
            double r2 = dth * dth / (m->theta_m * m->theta_m);
            Eb += -0.5 * kb * m->theta_m * m->theta_m * log(1.0 - r2);
            c = kb * dth / (1.0 - r2);
        } else {
            Eb += 0.5 * kb * dth * dth;
            c = kb * dth;
        }
        double ed[3], da[3], db[3], n1[3], n2[3], t1[3], t0[3], ta[3], tb[3];
        sub3(p1, p0, ed); sub3(pa, p0, da); sub3(pb, p0, db);
        cross3(ed, da, n1);
        cross3(db, ed, n2);
        double L = sqrt(dot3(ed, ed));
        double q1 = dot3(n1, n1), q2 = dot3(n2, n2);
        double pa1[3], pb1[3];
        sub3(pa, p1, pa1); sub3(pb, p1, pb1);
        double sa0 = dot3(pa1, ed) / L, sb0 = dot3(pb1, ed) / L; /* (pa-p1).e/L, (pb-p1).e/L */
        double sa1 = dot3(da, ed) / L, sb1 = dot3(db, ed) / L;   /* (pa-p0).e/L, (pb-p0).e/L */
        for (int k = 0; k < 3; ++k) {
            ta[k] = -L * n1[k] / q1;
            tb[k] = -L * n2[k] / q2;
            t0[k] = -sa0 * n1[k] / q1 - sb0 * n2[k] / q2;
            t1[k] = sa1 * n1[k] / q1 + sb1 * n2[k] / q2;
        }
        for (int k = 0; k < 3; ++k) {
            F[3 * E[0] + k] -= c * t0[k];
            F[3 * E[1] + k] -= c * t1[k];
            F[3 * E[2] + k] -= c * ta[k];
            F[3 * E[3] + k] -= c * tb[k];
        }
    }
    /* area and volume: per cell totals, then per triangle gradients */
    double A, V;
    cell_area_volume(m, X, &A, &V);
    Ea = 0.5 * m->k_area * (A - m->A0) * (A - m->A0) / (m->A0 * m->A0);
    Ev = 0.5 * m->k_volume * (V - m->V0) * (V - m->V0) / (m->V0 * m->V0);
    double ca = m->k_area * (A - m->A0) / (m->A0 * m->A0);
    double cv = m->k_volume * (V - m->V0) / (m->V0 * m->V0);
    double ctr[3] = {0, 0, 0};
    for (int v = 0; v < m->nv; ++v) for (int d = 0; d < 3; ++d) ctr[d] += X[3 * v + d];
    for (int d = 0; d < 3; ++d) ctr[d] /= m->nv;
    for (int t = 0; t < m->nt; ++t) {
        int i0 = m->tri[3 * t], i1 = m->tri[3 * t + 1], i2 = m->tri[3 * t + 2];
        const double *x0 = X + 3 * i0, *x1 = X + 3 * i1, *x2 = X + 3 * i2;
        double e1[3], e2[3], n[3];
        sub3(x1, x0, e1); sub3(x2, x0, e2); cross3(e1, e2, n);
        double nn = sqrt(dot3(n, n));
        double nh[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
        /* dE/dA_t of the global (per cell) and the local (per triangle) area terms */
        double ct = ca;
        if (m->k_local > 0) {
            double At = 0.5 * nn;
            Ea += 0.5 * m->k_local * (At - m->At0[t]) * (At - m->At0[t]) / m->At0[t];
            ct += m->k_local * (At - m->At0[t]) / m->At0[t];
        }
        double d21[3], d02[3], d10[3], g0[3], g1[3], g2[3];
        sub3(x2, x1, d21); sub3(x0, x2, d02); sub3(x1, x0, d10);
        cross3(nh, d21, g0); cross3(nh, d02, g1); cross3(nh, d10, g2);
        double r0[3], r1[3], r2[3], v0[3], v1[3], v2[3];
        sub3(x0, ctr, r0); sub3(x1, ctr, r1); sub3(x2, ctr, r2);
        cross3(r1, r2, v0); cross3(r2, r0, v1); cross3(r0, r1, v2);
        for (int k = 0; k < 3; ++k) {
            F[3 * i0 + k] -= ct * 0.5 * g0[k] + cv * v0[k] / 6.0;
            F[3 * i1 + k] -= ct * 0.5 * g1[k] + cv * v1[k] / 6.0;
            F[3 * i2 + k] -= ct * 0.5 * g2[k] + cv * v2[k] / 6.0;
        }
    }
    if (E4) { E4[0] = El; E4[1] = Eb; E4[2] = Ea; E4[3] = Ev; }
    if (Aout) *Aout = A;
    if (Vout) *Vout = V;
}

/* Standalone membrane evaluation for one cell (pins): rest shape + params,
 * positions X; writes forces F (nv*3, overwritten) and energies E4. */
int ora_membrane(int nv, int nt, const int *tri, const double *rest, const double *params,
                 const double *X, double *F, double *E4, double *AV) {
    omesh m;
    if (mesh_init(&m, nv, nt, tri, rest, params) < 0) { mesh_free(&m); return -1; }
    memset(F, 0, sizeof(double) * 3 * nv);
    double A, V;
    membrane_forces(&m, X, F, E4, &A, &V);
    if (AV) { AV[0] = A; AV[1] = V; AV[2] = m.A0; AV[3] = m.V0; }
    mesh_free(&m);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* simulation                                                                */
/* ------------------------------------------------------------------------ */
#define MAXTYPES 8
typedef struct {
    int nx, ny, nz;
    long N;
    double tau;
    int periodic[3];
    unsigned char *mask;   /* N */
    double uw[4][3];       /* wall velocity by mask id */
    double g[3];
    double *f, *fn;        /* N*Q */
    double *rho_c;         /* collision density, N */
    double *F;             /* N*3 */
    double *u;             /* N*3 */
    int ntypes;
    omesh types[MAXTYPES];
    int ncell;
    int *cell_type, *cell_first;
    long nvtot;
    double *X, *Fv;        /* nvtot*3 */
    double *X0c;           /* initial centroids, ncell*3 */
    double discarded[3];
    /* time-scale separation and vertex integrator (Sec. 2.6) */
    int force_every;       /* N >= 1 */
    int integrator;        /* ORA_EULER or ORA_AB2 */
    long nstep, ts_origin; /* steps taken; step at which the setting was made */
    int have_prev;         /* Up holds U^{n-1} */
    double *Up;            /* nvtot*3 */
    /* adaptive separation: re-evaluate when the largest vertex displacement
     * since the last evaluation exceeds adapt_delta (< 0: fixed schedule) */
    double adapt_delta;
    double *Xe;            /* nvtot*3 positions at the last evaluation */
    long last_eval;        /* step of the last evaluation, -1: none since the setting */
    long evaluations;      /* force evaluations so far */
    /* Lees-Edwards boundary along z */
    int le_on;
    double le_U;           /* velocity of the image above relative to the box */
    /* internal viscosity */
    double visc_ratio;     /* 1: off */
    unsigned char *inside; /* N, indicator of the current step */
    unsigned char *forced; /* N or NULL: indicator given by the caller (tests) */
} osim;

#define ORA_EULER 0
#define ORA_AB2 1

void *ora_create(int nx, int ny, int nz, double tau, const int *periodic, const unsigned char *mask,
                 const double *wall_velocity, const double *g) {
    build_tables();
    osim *s = (osim *)calloc(1, sizeof(osim));
    s->nx = nx; s->ny = ny; s->nz = nz;
    s->N = (long)nx * ny * nz;
    s->tau = tau;
    for (int d = 0; d < 3; ++d) s->periodic[d] = periodic[d];
    s->mask = (unsigned char *)calloc(s->N, 1);
    if (mask) memcpy(s->mask, mask, s->N);
    for (int d = 0; d < 3; ++d) {
        s->uw[0][d] = 0; s->uw[1][d] = 0;
        s->uw[2][d] = wall_velocity ? wall_velocity[d] : 0;
        s->uw[3][d] = wall_velocity ? wall_velocity[3 + d] : 0;
        s->g[d] = g ? g[d] : 0;
    }
    s->f = (double *)malloc(sizeof(double) * Q * s->N);
    s->fn = (double *)malloc(sizeof(double) * Q * s->N);
    s->rho_c = (double *)malloc(sizeof(double) * s->N);
    s->force_every = 1;
    s->integrator = ORA_EULER;
    s->adapt_delta = -1.0;
    s->last_eval = -1;
    s->visc_ratio = 1.0;
    s->inside = (unsigned char *)calloc(s->N, 1);
    s->F = (double *)calloc(3 * s->N, sizeof(double));
    s->u = (double *)calloc(3 * s->N, sizeof(double));
    for (long n = 0; n < s->N; ++n) {
        for (int i = 0; i < Q; ++i) s->f[n * Q + i] = s->fn[n * Q + i] = W[i];  /* (wall nodes keep w) */
        if (s->mask[n]) for (int d = 0; d < 3; ++d) s->u[3 * n + d] = s->uw[s->mask[n]][d];
    }
    return s;
}

void ora_destroy(void *p) {
    osim *s = (osim *)p;
    if (!s) return;
    for (int t = 0; t < s->ntypes; ++t) mesh_free(&s->types[t]);
    free(s->mask); free(s->f); free(s->fn); free(s->rho_c); free(s->F); free(s->u);
    free(s->cell_type); free(s->cell_first); free(s->X); free(s->Fv); free(s->X0c); free(s->Up); free(s->Xe);
    free(s->inside); free(s->forced);
    free(s);
}

int ora_add_mesh(void *p, int nv, int nt, const int *tri, const double *rest, const double *params) {
    osim *s = (osim *)p;
    if (s->ntypes >= MAXTYPES) return -1;
    if (mesh_init(&s->types[s->ntypes], nv, nt, tri, rest, params) < 0) return -1;
    return s->ntypes++;
}

static void centroid(const double *X, int nv, double *c) {
    c[0] = c[1] = c[2] = 0;
    for (int v = 0; v < nv; ++v) for (int d = 0; d < 3; ++d) c[d] += X[3 * v + d];
    for (int d = 0; d < 3; ++d) c[d] /= nv;
}

/* cells of one type: vertices = R * rest + center */
int ora_add_cells(void *p, int type, int ncell, const double *centers, const double *rots, const double *rest) {
    osim *s = (osim *)p;
    if (type < 0 || type >= s->ntypes) return -1;
    int nv = s->types[type].nv;
    long old = s->nvtot;
    s->cell_type = (int *)realloc(s->cell_type, sizeof(int) * (s->ncell + ncell));
    s->cell_first = (int *)realloc(s->cell_first, sizeof(int) * (s->ncell + ncell));
    s->X0c = (double *)realloc(s->X0c, sizeof(double) * 3 * (s->ncell + ncell));
    s->X = (double *)realloc(s->X, sizeof(double) * 3 * (old + (long)ncell * nv));
    s->Fv = (double *)realloc(s->Fv, sizeof(double) * 3 * (old + (long)ncell * nv));
    s->Up = (double *)realloc(s->Up, sizeof(double) * 3 * (old + (long)ncell * nv));
    if (s->Xe) s->Xe = (double *)realloc(s->Xe, sizeof(double) * 3 * (old + (long)ncell * nv));
    s->have_prev = 0;
    for (int c = 0; c < ncell; ++c) {
        int id = s->ncell + c;
        s->cell_type[id] = type;
        s->cell_first[id] = (int)(old + (long)c * nv);
        const double *R = rots + 9 * c;
        for (int v = 0; v < nv; ++v) {
            double *x = s->X + 3 * (old + (long)c * nv + v);
            for (int d = 0; d < 3; ++d)
                x[d] = centers[3 * c + d] + R[3 * d] * rest[3 * v] + R[3 * d + 1] * rest[3 * v + 1] + R[3 * d + 2] * rest[3 * v + 2];
            s->Fv[3 * (old + (long)c * nv + v)] = 0;
            s->Fv[3 * (old + (long)c * nv + v) + 1] = 0;
            s->Fv[3 * (old + (long)c * nv + v) + 2] = 0;
        }
        centroid(s->X + 3 * (old + (long)c * nv), nv, s->X0c + 3 * id);
    }
    s->ncell += ncell;
    s->nvtot = old + (long)ncell * nv;
    return 0;
}

void ora_set_vertices(void *p, const double *X) {
    osim *s = (osim *)p;
    memcpy(s->X, X, sizeof(double) * 3 * s->nvtot);
    s->have_prev = 0;
    s->ts_origin = s->nstep;
    s->last_eval = -1;
}

/* time-scale separation N (membrane forces every N steps, held in between)
 * and the vertex integrator; both count from the current step (Sec. 2.6) */
int ora_set_time_scales(void *p, int force_every, int integrator) {
    osim *s = (osim *)p;
    if (force_every < 1 || (integrator != ORA_EULER && integrator != ORA_AB2)) return -1;
    s->force_every = force_every;
    s->integrator = integrator;
    s->ts_origin = s->nstep;
    s->last_eval = -1;
    s->have_prev = 0;
    return 0;
}

/* Adaptive separation (Sec. 2.6: the separation may be adaptive; the
 * criterion of the cited work is not available, this is the build's own):
 * with delta >= 0 the membrane forces are evaluated on the first step after
 * this call, and then on every step at whose start the largest vertex
 * displacement |X_v - X_v(last evaluation)| exceeds delta, or at which
 * force_every steps have passed since the last evaluation; they are held
 * in between.  delta < 0: the constant schedule of ora_set_time_scales. */
int ora_set_force_tolerance(void *p, double delta) {
    osim *s = (osim *)p;
    if (delta != delta) return -1;
    s->adapt_delta = delta;
    s->last_eval = -1;
    s->ts_origin = s->nstep;
    if (delta >= 0 && !s->Xe) s->Xe = (double *)calloc(3 * (size_t)(s->nvtot > 0 ? s->nvtot : 1), sizeof(double));
    return 0;
}

long ora_force_evaluations(void *p) { return ((osim *)p)->evaluations; }

/* whether the membrane forces are evaluated on the current step */
static int force_step(osim *s) {
    if (s->adapt_delta < 0) return (s->nstep - s->ts_origin) % s->force_every == 0;
    if (s->last_eval < 0 || s->nstep - s->last_eval >= s->force_every) return 1;
    double m2 = 0;
    for (long k = 0; k < s->nvtot; ++k) {
        double d2 = 0;
        for (int d = 0; d < 3; ++d) {
            const double e = s->X[3 * k + d] - s->Xe[3 * k + d];
            d2 += e * e;
        }
        if (d2 > m2) m2 = d2;
    }
    return sqrt(m2) > s->adapt_delta;
}

/* populations at equilibrium with rho = 1 and the given velocity field
 * (N*3, NULL = rest) */
void ora_set_velocity(void *p, const double *u0) {
    osim *s = (osim *)p;
    for (long n = 0; n < s->N; ++n) {
        if (s->mask[n]) continue;
        double u[3] = {0, 0, 0};
        if (u0) { u[0] = u0[3 * n]; u[1] = u0[3 * n + 1]; u[2] = u0[3 * n + 2]; }
        ora_equilibrium(1.0, u, s->f + n * Q);
        for (int d = 0; d < 3; ++d) s->u[3 * n + d] = u[d];
    }
}

/* neighbour of node (x,y,z) along c; returns -1 outside a non-periodic axis */
static long neighbour(const osim *s, int x, int y, int z, int cx, int cy, int cz) {
    int xx = x + cx, yy = y + cy, zz = z + cz;
    int dims[3] = {s->nx, s->ny, s->nz};
    int q[3] = {xx, yy, zz};
    for (int d = 0; d < 3; ++d) {
        if (q[d] < 0 || q[d] >= dims[d]) {
            if (!s->periodic[d]) return -1;
            q[d] = ((q[d] % dims[d]) + dims[d]) % dims[d];
        }
    }
    return q[0] + (long)s->nx * (q[1] + (long)s->ny * q[2]);
}

/* ---- inside/outside indicator (internal viscosity) ------------------- */
/* twice the signed area of the xy-projection, edge u -> v against point p,
 * always computed from the lower-numbered vertex so that the two triangles
 * of an edge get exactly opposite values */
static double edge_fn(const double *X, int iu, int iv, double px, double py) {
    if (iu < iv) {
        const double *u = X + 3 * iu, *v = X + 3 * iv;
        return (v[0] - u[0]) * (py - u[1]) - (v[1] - u[1]) * (px - u[0]);
    }
    const double *u = X + 3 * iv, *v = X + 3 * iu;
    return -((v[0] - u[0]) * (py - u[1]) - (v[1] - u[1]) * (px - u[0]));
}

/* does the xy-projection of triangle (i0, i1, i2) (positions X) contain
 * (px, py)?  sgn receives the sign of the outward normal's z component, zc
 * the height of the triangle's plane at (px, py) */
static int tri_column(const double *X, int i0, int i1, int i2, double px, double py, int *sgn, double *zc) {
    const double *a = X + 3 * i0, *b = X + 3 * i1, *c = X + 3 * i2;
    double e1[3], e2[3], n[3];
    sub3(b, a, e1); sub3(c, a, e2); cross3(e1, e2, n);
    if (n[2] == 0) return 0;
    /* counter-clockwise seen from +z */
    int v[3] = {i0, i1, i2};
    if (n[2] < 0) { v[1] = i2; v[2] = i1; }
    for (int k = 0; k < 3; ++k) {
        int iu = v[k], iv = v[(k + 1) % 3];
        double e = edge_fn(X, iu, iv, px, py);
        if (e < 0) return 0;
        if (e == 0) {
            double dx = X[3 * iv] - X[3 * iu], dy = X[3 * iv + 1] - X[3 * iu + 1];
            if (!(dy < 0 || (dy == 0 && dx > 0))) return 0;
        }
    }
    *sgn = n[2] > 0 ? 1 : -1;
    *zc = a[2] - (n[0] * (px - a[0]) + n[1] * (py - a[1])) / n[2];
    return 1;
}

/* indicator of the current vertex positions: per cell, every node of the
 * lattice within the bounding box of the cell or of one of its periodic
 * images sums, over the triangles whose projection contains its column,
 * the signs of the crossings above it */
static void compute_inside(osim *s, unsigned char *in) {
    memset(in, 0, s->N);
    const long dims[3] = {s->nx, s->ny, s->nz};
    for (int c = 0; c < s->ncell; ++c) {
        const omesh *m = &s->types[s->cell_type[c]];
        const double *X = s->X + 3 * (long)s->cell_first[c];
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) { lo[d] = X[d]; hi[d] = X[d]; }
        for (int v = 1; v < m->nv; ++v)
            for (int d = 0; d < 3; ++d) {
                if (X[3 * v + d] < lo[d]) lo[d] = X[3 * v + d];
                if (X[3 * v + d] > hi[d]) hi[d] = X[3 * v + d];
            }
        int kmin[3], kmax[3];
        for (int d = 0; d < 3; ++d) { kmin[d] = s->periodic[d] ? -1 : 0; kmax[d] = s->periodic[d] ? 1 : 0; }
        for (int kx = kmin[0]; kx <= kmax[0]; ++kx)
            for (int ky = kmin[1]; ky <= kmax[1]; ++ky)
                for (int kz = kmin[2]; kz <= kmax[2]; ++kz) {
                    const long k[3] = {kx, ky, kz};
                    long j0[3], j1[3];
                    int empty = 0;
                    for (int d = 0; d < 3; ++d) {
                        j0[d] = (long)ceil(lo[d] + k[d] * dims[d]);
                        j1[d] = (long)floor(hi[d] + k[d] * dims[d]);
                        if (j0[d] < 0) j0[d] = 0;
                        if (j1[d] > dims[d] - 1) j1[d] = dims[d] - 1;
                        if (j0[d] > j1[d]) empty = 1;
                    }
                    if (empty) continue;
                    for (long jz = j0[2]; jz <= j1[2]; ++jz)
                        for (long jy = j0[1]; jy <= j1[1]; ++jy)
                            for (long jx = j0[0]; jx <= j1[0]; ++jx) {
                                /* the node in the cell's own (unwrapped) frame */
                                double px = (double)(jx - kx * dims[0]), py = (double)(jy - ky * dims[1]);
                                double pz = (double)(jz - kz * dims[2]);
                                int w = 0;
                                for (int t = 0; t < m->nt; ++t) {
                                    int sg;
                                    double zc;
                                    if (tri_column(X, m->tri[3 * t], m->tri[3 * t + 1], m->tri[3 * t + 2], px, py, &sg, &zc)
                                        && zc > pz)
                                        w += sg;
                                }
                                if (w != 0) in[jx + s->nx * (jy + s->ny * jz)] = 1;
                            }
                }
    }
}

/* indicator at the current positions (N bytes) */
void ora_inside(void *p, unsigned char *out) {
    compute_inside((osim *)p, out);
}

/* internal viscosity ratio (1 = off) */
int ora_set_viscosity_ratio(void *p, double ratio) {
    if (!(ratio > 0)) return -1;
    if (((osim *)p)->le_on && ratio != 1.0) return -1;  /* the rays would cross the displaced plane */
    ((osim *)p)->visc_ratio = ratio;
    return 0;
}

/* Lees-Edwards boundary with image velocity U (before the first step; needs
 * a fully periodic lattice without walls) */
int ora_set_lees_edwards(void *p, double U) {
    osim *s = (osim *)p;
    if (s->nstep != 0) return -1;
    for (int d = 0; d < 3; ++d) if (!s->periodic[d]) return -1;
    for (long n = 0; n < s->N; ++n) if (s->mask[n]) return -1;
    if (s->visc_ratio != 1.0) return -1;
    s->le_on = 1;
    s->le_U = U;
    return 0;
}

/* image displacement of the current step, in [0, nx) */
static double le_shift(const osim *s) {
    double D = fmod(s->le_U * (double)s->nstep, (double)s->nx);
    return D < 0 ? D + s->nx : D;
}

/* tests: take the indicator from the caller (N bytes) instead of the cells;
 * NULL returns to the computed one */
void ora_force_inside(void *p, const unsigned char *ind) {
    osim *s = (osim *)p;
    free(s->forced);
    s->forced = NULL;
    if (ind) {
        s->forced = (unsigned char *)malloc(s->N);
        memcpy(s->forced, ind, s->N);
    }
}

/* node index of lattice coordinate j along each axis, -1 if outside */
static long node_at(const osim *s, long jx, long jy, long jz) {
    long q[3] = {jx, jy, jz};
    long dims[3] = {s->nx, s->ny, s->nz};
    for (int d = 0; d < 3; ++d) {
        if (q[d] < 0 || q[d] >= dims[d]) {
            if (!s->periodic[d]) return -1;
            q[d] = ((q[d] % dims[d]) + dims[d]) % dims[d];
        }
    }
    return q[0] + s->nx * (q[1] + s->ny * q[2]);
}

/* Per fluid node: bit i set when node + c_i is a wall or outside a
 * non-periodic axis (oracle's velocity order); 0 at wall nodes. */
void ora_wall_links(void *p, uint32_t *links) {
    osim *s = (osim *)p;
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long n = x + (long)s->nx * (y + (long)s->ny * z);
                uint32_t b = 0;
                if (!s->mask[n])
                    for (int i = 0; i < Q; ++i) {
                        long m = neighbour(s, x, y, z, C[i][0], C[i][1], C[i][2]);
                        if (m < 0 || s->mask[m]) b |= 1u << i;
                    }
                links[n] = b;
            }
}

/* one coupled step, Sec. 2.3 order: forces at X^n, spread, collide+stream,
 * velocity, interpolate and move */
static void step_once(osim *s) {
    const long N = s->N;
    const double D = s->le_on ? le_shift(s) : 0.0;
    /* 0: Lees-Edwards: cells whose centroid left the box through the sheared
     * plane move to the other side */
    if (s->le_on)
        for (int c = 0; c < s->ncell; ++c) {
            const omesh *m = &s->types[s->cell_type[c]];
            double *X = s->X + 3 * (long)s->cell_first[c];
            double ctr[3];
            centroid(X, m->nv, ctr);
            double dx = 0, dz = 0;
            if (ctr[2] >= s->nz) { dx = -D; dz = -s->nz; }
            else if (ctr[2] < 0) { dx = D; dz = s->nz; }
            if (dz != 0)
                for (int v = 0; v < m->nv; ++v) { X[3 * v] += dx; X[3 * v + 2] += dz; }
        }
    /* 1-2: membrane forces at the current positions (per cell), on every
     * N-th step only; the last ones are held in between */
    if (force_step(s)) {
        if (s->adapt_delta >= 0) {
            memcpy(s->Xe, s->X, sizeof(double) * 3 * s->nvtot);
            s->last_eval = s->nstep;
        }
        s->evaluations += 1;
        for (long v = 0; v < 3 * s->nvtot; ++v) s->Fv[v] = 0;
        #pragma omp parallel for schedule(static)
        for (int c = 0; c < s->ncell; ++c) {
            const omesh *m = &s->types[s->cell_type[c]];
            long o = s->cell_first[c];
            membrane_forces(m, s->X + 3 * o, s->Fv + 3 * o, NULL, NULL, NULL);
        }
    }
    /* 3: F(x) = g + sum_v F_v delta_h(x - X_v); wall nodes discard */
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n)
        for (int d = 0; d < 3; ++d) s->F[3 * n + d] = s->mask[n] ? 0.0 : s->g[d];
    s->discarded[0] = s->discarded[1] = s->discarded[2] = 0;
    for (long v = 0; v < s->nvtot; ++v) {
        const double *X = s->X + 3 * v;
        long i0[3];
        for (int d = 0; d < 3; ++d) i0[d] = (long)floor(X[d]);
        for (int c = -1; c <= 2; ++c) {
            long jz = i0[2] + c;
            /* Lees-Edwards: a layer in the image above (below) takes the
             * position displaced by -D (+D) */
            double xp = X[0];
            if (s->le_on && jz >= s->nz) xp = X[0] - D;
            else if (s->le_on && jz < 0) xp = X[0] + D;
            long ix = (long)floor(xp);
            for (int a = -1; a <= 2; ++a)
                for (int b = -1; b <= 2; ++b) {
                    long jx = ix + a, jy = i0[1] + b;
                    double dl = ora_phi(xp - jx) * ora_phi(X[1] - jy) * ora_phi(X[2] - jz);
                    long n = node_at(s, jx, jy, jz);
                    for (int d = 0; d < 3; ++d) {
                        double add = s->Fv[3 * v + d] * dl;
                        if (n >= 0 && !s->mask[n]) s->F[3 * n + d] += add;
                        else s->discarded[d] += add;
                    }
                }
        }
    }
    /* 4: BGK collision with the Guo forcing term (in place in f); inside
     * cells tau_in = 1/2 + lambda (tau - 1/2) */
    const double om_out = 1.0 / s->tau, om_in = 1.0 / (0.5 + s->visc_ratio * (s->tau - 0.5));
    const int contrast = s->visc_ratio != 1.0;
    if (contrast) {
        if (s->forced) memcpy(s->inside, s->forced, N);
        else compute_inside(s, s->inside);
    }
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->mask[n]) continue;
        const double om = contrast && s->inside[n] ? om_in : om_out;
        double *f = s->f + n * Q;
        const double *Fn = s->F + 3 * n;
        double rho = 0, m[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            rho += f[i];
            for (int d = 0; d < 3; ++d) m[d] += f[i] * C[i][d];
        }
        double u[3];
        for (int d = 0; d < 3; ++d) u[d] = (m[d] + 0.5 * Fn[d]) / rho;
        double feq[Q];
        ora_equilibrium(rho, u, feq);
        for (int i = 0; i < Q; ++i) {
            double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
            double Si = 0;
            for (int d = 0; d < 3; ++d) Si += (3.0 * (C[i][d] - u[d]) + 9.0 * cu * C[i][d]) * Fn[d];
            Si *= (1.0 - 0.5 * om) * W[i];
            f[i] = f[i] - om * (f[i] - feq[i]) + Si;
        }
        s->rho_c[n] = rho;
    }
    /* 5: pull streaming with halfway bounce-back */
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long n = x + (long)s->nx * (y + (long)s->ny * z);
                if (s->mask[n]) continue;
                for (int i = 0; i < Q; ++i) {
                    int zs = z - C[i][2];
                    if (s->le_on && (zs < 0 || zs >= s->nz)) {
                        /* from the image above (zs = nz) or below (zs = -1) */
                        int up = zs >= s->nz;
                        double xs = x - C[i][0] + (up ? -D : D);
                        long xa = (long)floor(xs);
                        double wb = xs - xa;
                        int ys = y - C[i][1], zb = up ? 0 : s->nz - 1;
                        double val = 0;
                        for (int k = 0; k < 2; ++k) {
                            long sn = node_at(s, xa + k, ys, zb);
                            const double *fs = s->f + sn * Q;
                            double r = 0, mm[3] = {0, 0, 0};
                            for (int j = 0; j < Q; ++j) {
                                r += fs[j];
                                for (int d = 0; d < 3; ++d) mm[d] += fs[j] * C[j][d];
                            }
                            double us[3] = {mm[0] / r, mm[1] / r, mm[2] / r}, ush[3] = {us[0] + (up ? s->le_U : -s->le_U), us[1], us[2]};
                            double e0[Q], e1[Q];
                            ora_equilibrium(r, us, e0);
                            ora_equilibrium(r, ush, e1);
                            val += (k ? wb : 1.0 - wb) * (fs[i] + (e1[i] - e0[i]));
                        }
                        s->fn[n * Q + i] = val;
                        continue;
                    }
                    long src = neighbour(s, x, y, z, -C[i][0], -C[i][1], -C[i][2]);
                    if (src >= 0 && !s->mask[src]) {
                        s->fn[n * Q + i] = s->f[src * Q + i];
                    } else {
                        int j = OPP[i];
                        const double *uw = s->uw[src >= 0 ? s->mask[src] : 1];
                        double cu = C[j][0] * uw[0] + C[j][1] * uw[1] + C[j][2] * uw[2];
                        s->fn[n * Q + i] = s->f[n * Q + j] - 6.0 * W[j] * s->rho_c[n] * cu;
                    }
                }
            }
    double *tmp = s->f; s->f = s->fn; s->fn = tmp;
    /* 6: velocity of the streamed populations with the applied force F/2 */
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->mask[n]) continue;
        const double *f = s->f + n * Q;
        double rho = 0, m[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            rho += f[i];
            for (int d = 0; d < 3; ++d) m[d] += f[i] * C[i][d];
        }
        for (int d = 0; d < 3; ++d) s->u[3 * n + d] = (m[d] + 0.5 * s->F[3 * n + d]) / rho;
    }
    /* 7: interpolate U^n at X^n and move (dt = 1): Euler X += U^n, or
     * Adams-Bashforth X += 3/2 U^n - 1/2 U^{n-1} once U^{n-1} exists */
    const int ab2 = s->integrator == ORA_AB2 && s->have_prev;
    #pragma omp parallel for schedule(static)
    for (long v = 0; v < s->nvtot; ++v) {
        double *X = s->X + 3 * v;
        long i0[3];
        for (int d = 0; d < 3; ++d) i0[d] = (long)floor(X[d]);
        double U[3] = {0, 0, 0};
        for (int c = -1; c <= 2; ++c) {
            long jz = i0[2] + c;
            /* Lees-Edwards: a layer in the image above (below) takes the
             * displaced position and the image's velocity +U (-U) */
            double xp = X[0], du = 0;
            if (s->le_on && jz >= s->nz) { xp = X[0] - D; du = s->le_U; }
            else if (s->le_on && jz < 0) { xp = X[0] + D; du = -s->le_U; }
            long ix = (long)floor(xp);
            for (int a = -1; a <= 2; ++a)
                for (int b = -1; b <= 2; ++b) {
                    long jx = ix + a, jy = i0[1] + b;
                    double dl = ora_phi(xp - jx) * ora_phi(X[1] - jy) * ora_phi(X[2] - jz);
                    long n = node_at(s, jx, jy, jz);
                    if (n < 0) continue; /* resting wall outside the domain */
                    U[0] += (s->u[3 * n] + du) * dl;
                    U[1] += s->u[3 * n + 1] * dl;
                    U[2] += s->u[3 * n + 2] * dl;
                }
        }
        double *Up = s->Up + 3 * v;
        for (int d = 0; d < 3; ++d) {
            X[d] += ab2 ? 1.5 * U[d] - 0.5 * Up[d] : U[d];
            Up[d] = U[d];
        }
    }
    s->have_prev = s->integrator == ORA_AB2;
    s->nstep += 1;
}

/* worker threads of the annotated loops (no effect without OpenMP) */
void ora_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int ora_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_step(void *p, int nsteps) {
    osim *s = (osim *)p;
    for (int k = 0; k < nsteps; ++k) step_once(s);
}

/* density of the current populations (N), velocity field (N*3), vertices
 * (nvtot*3), last membrane forces (nvtot*3), per-cell stats (ncell*6:
 * centroid, area, volume, deformation index) at the current positions. */
static double deformation_index(const double *X, int nv);

void ora_get(void *p, double *rho, double *u, double *X, double *Fv, double *cellstats, double *discarded) {
    osim *s = (osim *)p;
    if (rho)
        for (long n = 0; n < s->N; ++n) {
            double r = 0;
            if (!s->mask[n]) for (int i = 0; i < Q; ++i) r += s->f[n * Q + i];
            rho[n] = s->mask[n] ? 0.0 : r;
        }
    if (u) memcpy(u, s->u, sizeof(double) * 3 * s->N);
    if (X) memcpy(X, s->X, sizeof(double) * 3 * s->nvtot);
    if (Fv) memcpy(Fv, s->Fv, sizeof(double) * 3 * s->nvtot);
    if (cellstats)
        for (int c = 0; c < s->ncell; ++c) {
            const omesh *m = &s->types[s->cell_type[c]];
            const double *Xc = s->X + 3 * (long)s->cell_first[c];
            double ctr[3], A, V;
            centroid(Xc, m->nv, ctr);
            cell_area_volume(m, Xc, &A, &V);
            double *o = cellstats + 6 * c;
            o[0] = ctr[0]; o[1] = ctr[1]; o[2] = ctr[2]; o[3] = A; o[4] = V;
            o[5] = deformation_index(Xc, m->nv);
        }
    if (discarded) for (int d = 0; d < 3; ++d) discarded[d] = s->discarded[d];
}

/* raw populations, oracle order, N*Q */
void ora_get_populations(void *p, double *f) {
    osim *s = (osim *)p;
    memcpy(f, s->f, sizeof(double) * Q * s->N);
}

/* ------------------------------------------------------------------------ */
/* coupling operators alone (pins): spread F_v -> F and interpolate u -> U   */
/* ------------------------------------------------------------------------ */
void ora_spread(void *p, long nv, const double *X, const double *Fv, double *F_out) {
    osim *s = (osim *)p;
    memset(F_out, 0, sizeof(double) * 3 * s->N);
    for (long v = 0; v < nv; ++v) {
        const double *x = X + 3 * v;
        long i0[3];
        for (int d = 0; d < 3; ++d) i0[d] = (long)floor(x[d]);
        for (int a = -1; a <= 2; ++a)
            for (int b = -1; b <= 2; ++b)
                for (int c = -1; c <= 2; ++c) {
                    long jx = i0[0] + a, jy = i0[1] + b, jz = i0[2] + c;
                    double dl = ora_phi(x[0] - jx) * ora_phi(x[1] - jy) * ora_phi(x[2] - jz);
                    long n = node_at(s, jx, jy, jz);
                    if (n < 0 || s->mask[n]) continue;
                    for (int d = 0; d < 3; ++d) F_out[3 * n + d] += Fv[3 * v + d] * dl;
                }
    }
}

void ora_interpolate(void *p, long nv, const double *X, const double *u, double *U) {
    osim *s = (osim *)p;
    for (long v = 0; v < nv; ++v) {
        const double *x = X + 3 * v;
        long i0[3];
        for (int d = 0; d < 3; ++d) i0[d] = (long)floor(x[d]);
        U[3 * v] = U[3 * v + 1] = U[3 * v + 2] = 0;
        for (int a = -1; a <= 2; ++a)
            for (int b = -1; b <= 2; ++b)
                for (int c = -1; c <= 2; ++c) {
                    long jx = i0[0] + a, jy = i0[1] + b, jz = i0[2] + c;
                    double dl = ora_phi(x[0] - jx) * ora_phi(x[1] - jy) * ora_phi(x[2] - jz);
                    long n = node_at(s, jx, jy, jz);
                    if (n < 0) continue;
                    for (int d = 0; d < 3; ++d) U[3 * v + d] += u[3 * n + d] * dl;
                }
    }
}

/* ------------------------------------------------------------------------ */
/* vertex binning: key = lattice block of floor(X) (wrapped on periodic     */
/* axes, clamped otherwise); stable counting sort by key                    */
/* ------------------------------------------------------------------------ */
int ora_bins(void *p, long nv, const double *X, int B, int32_t *key, int32_t *perm, int32_t *start) {
    osim *s = (osim *)p;
    int dims[3] = {s->nx, s->ny, s->nz};
    int nb[3];
    for (int d = 0; d < 3; ++d) nb[d] = (dims[d] + B - 1) / B;
    long nbins = (long)nb[0] * nb[1] * nb[2];
    for (long v = 0; v < nv; ++v) {
        int b[3];
        for (int d = 0; d < 3; ++d) {
            long j = (long)floor(X[3 * v + d]);
            if (s->periodic[d]) j = ((j % dims[d]) + dims[d]) % dims[d];
            else j = j < 0 ? 0 : (j >= dims[d] ? dims[d] - 1 : j);
            b[d] = (int)(j / B);
        }
        key[v] = (int32_t)(b[0] + (long)nb[0] * (b[1] + (long)nb[1] * b[2]));
    }
    for (long k = 0; k <= nbins; ++k) start[k] = 0;
    for (long v = 0; v < nv; ++v) start[key[v] + 1]++;
    for (long k = 0; k < nbins; ++k) start[k + 1] += start[k];
    int32_t *cursor = (int32_t *)malloc(sizeof(int32_t) * nbins);
    for (long k = 0; k < nbins; ++k) cursor[k] = start[k];
    for (long v = 0; v < nv; ++v) perm[cursor[key[v]]++] = (int32_t)v;
    free(cursor);
    return (int)nbins;
}

/* ------------------------------------------------------------------------ */
/* deformation loss (differentiation form)                                  */
/* ------------------------------------------------------------------------ */
/* eigenvalues of a symmetric 3x3 matrix by cyclic Jacobi rotations */
static void sym3_eigenvalues(double a[3][3], double ev[3]) {
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        if (off < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) { /* columns p, q */
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - sn * akq;
                    a[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) { /* rows p, q */
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - sn * aqk;
                    a[q][k] = sn * apk + c * aqk;
                }
            }
    }
    ev[0] = a[0][0]; ev[1] = a[1][1]; ev[2] = a[2][2];
}

/* Taylor deformation index from the gyration tensor G = mean (X-c)(X-c)^T:
 * DI = (sqrt(l1) - sqrt(l3)) / (sqrt(l1) + sqrt(l3)), l1 >= l2 >= l3 */
static double deformation_index(const double *X, int nv) {
    double c[3];
    centroid(X, nv, c);
    double G[3][3] = {{0}};
    for (int v = 0; v < nv; ++v) {
        double r[3];
        sub3(X + 3 * v, c, r);
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) G[i][j] += r[i] * r[j] / nv;
    }
    double ev[3];
    sym3_eigenvalues(G, ev);
    double lmax = ev[0], lmin = ev[0];
    for (int i = 1; i < 3; ++i) { if (ev[i] > lmax) lmax = ev[i]; if (ev[i] < lmin) lmin = ev[i]; }
    double a = sqrt(lmax), b = sqrt(lmin > 0 ? lmin : 0);
    return (a - b) / (a + b);
}

double ora_deformation_index(const double *X, int nv) { return deformation_index(X, nv); }

/* loss = mean_c DI_c + mean_c |centroid_c - initial centroid_c|^2 */
double ora_loss(void *p) {
    osim *s = (osim *)p;
    double di = 0, drift = 0;
    for (int c = 0; c < s->ncell; ++c) {
        const omesh *m = &s->types[s->cell_type[c]];
        const double *Xc = s->X + 3 * (long)s->cell_first[c];
        double ctr[3];
        centroid(Xc, m->nv, ctr);
        di += deformation_index(Xc, m->nv);
        for (int d = 0; d < 3; ++d) drift += (ctr[d] - s->X0c[3 * c + d]) * (ctr[d] - s->X0c[3 * c + d]);
    }
    return s->ncell ? (di + drift) / s->ncell : 0.0;
}

long ora_num_vertices(void *p) { return ((osim *)p)->nvtot; }
int ora_num_cells(void *p) { return ((osim *)p)->ncell; }
