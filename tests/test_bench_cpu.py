"""Host logic of bench.py that its JSON line rests on, without a GPU: the
algorithmic bytes per fluid node of the collision, the DRAM traffic record
that is reported only while the lattice source it was captured from is
unchanged, and the summary of the sampled clocks and throttle reasons."""
import json
import os
import shutil

import bench


def test_collision_bytes_per_node():
    # 19 populations read and 19 written at S bytes, plus the force density
    # (3 components at the arithmetic type's size)
    assert bench.bytes_per_node('f64') == 38 * 8 + 3 * 8
    assert bench.bytes_per_node('f32') == 38 * 4 + 3 * 4 == 164
    assert bench.bytes_per_node('f16') == bench.bytes_per_node('bf16') == 38 * 2 + 3 * 4 == 88


def _tree(tmp_path):
    root = tmp_path / 'repo'
    csrc = root / 'paper_2305_02752_gb300' / 'csrc'
    csrc.mkdir(parents=True)
    for f in ('k_lattice.cu', 'lattice_core.cuh'):
        shutil.copy(os.path.join(bench.ROOT, 'paper_2305_02752_gb300', 'csrc', f), csrc / f)
    shutil.copytree(os.path.join(bench.ROOT, 'profiles'), root / 'profiles')
    return root


def test_traffic_record_follows_the_lattice_source(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, 'ROOT', str(root))
    rec = json.load(open(root / 'profiles' / 'collide_f32_pipe.json'))
    assert bench.traffic_from_profile('f32', 'pipe') == rec['dram_bytes_per_launch']
    # the record is within 1 % of the algorithmic bytes it was checked against
    assert abs(rec['dram_bytes_per_launch'] / rec['algorithmic_bytes_per_launch'] - 1) < 0.01
    assert bench.traffic_from_profile('f32', 'vessel') is None  # no record for that workload
    with open(root / 'paper_2305_02752_gb300' / 'csrc' / 'k_lattice.cu', 'a') as f:
        f.write('\n// changed\n')
    assert bench.traffic_from_profile('f32', 'pipe') is None  # the kernel changed since the capture


def test_clock_summary():
    line = '0, {sm}, 2070, 900.5, 0x{a:x}, {hw}, Not Active, Not Active, {cap}\n'
    lines = [line.format(sm=2070, a=0, hw='Not Active', cap='Not Active'),
             line.format(sm=1980, a=4, hw='Not Active', cap='Active'),
             line.format(sm=2055, a=0, hw='Not Active', cap='Not Active'),
             '0, [N/A], 2070\n',  # incomplete line
             line.format(sm='[N/A]', a=0, hw='Not Active', cap='Not Active')]
    out = bench.ClockSampler.summarise(lines)
    assert out['samples'] == 4
    assert out['sm_mhz'] == 2055.0 and out['sm_max_mhz'] == 2070.0
    assert out['reasons'] == ['sw_power_cap']
    out = bench.ClockSampler.summarise([line.format(sm=1500, a=8, hw='Active', cap='Not Active')])
    assert out['reasons'] == ['hw_slowdown'] and out['sm_mhz'] == 1500.0
    assert bench.ClockSampler.summarise([]) == {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': [], 'samples': 0}
