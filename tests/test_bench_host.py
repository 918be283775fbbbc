"""Host-side pieces of the benchmark (CPU): the committed DRAM-traffic records belong to the current
kernel sources, a changed source drops them, and the shock workload shards like the plain one."""
import hashlib
import os

import numpy as np

import bench
from paper_1809_05608_gb300 import problems


def test_traffic_records_match_the_current_kernel_sources():
    """bench.py reports roofline traffic only while the sources hash to the digest of the ncu
    capture; the committed records must be those of the committed sources."""
    for kernel in ('k_assemble', 'k_factor', 'k_factor_row2', 'k_solve_tma', 'k_resid_ff'):
        rec = bench.traffic_record(kernel)
        assert rec is not None and rec['bytes'] > 0 and rec['units'] == 256.0, kernel


def test_a_changed_source_drops_the_traffic_record(tmp_path, monkeypatch):
    root = tmp_path / 'repo'
    (root / 'profiles').mkdir(parents=True)
    (root / 'paper_1809_05608_gb300' / 'csrc').mkdir(parents=True)
    csrc = os.path.join(bench.ROOT, 'paper_1809_05608_gb300', 'csrc')
    for name in ('blocktri.cu', 'assemble.cu'):
        data = open(os.path.join(csrc, name), 'rb').read()
        (root / 'paper_1809_05608_gb300' / 'csrc' / name).write_bytes(data + (b'\n' if name == 'assemble.cu' else b''))
    (root / 'profiles' / 'ncu_traffic.txt').write_text(
        open(os.path.join(bench.ROOT, 'profiles', 'ncu_traffic.txt')).read())
    monkeypatch.setattr(bench, 'ROOT', str(root))
    assert bench.traffic_record('k_assemble') is None
    src = (root / 'paper_1809_05608_gb300' / 'csrc' / 'blocktri.cu').read_bytes()
    src += (root / 'paper_1809_05608_gb300' / 'csrc' / 'assemble.cu').read_bytes()
    digest = hashlib.sha256(src).hexdigest()[:16]
    with open(root / 'profiles' / 'ncu_traffic.txt', 'a') as f:
        f.write(f'k_assemble       123   4      {digest}\n')
    assert bench.traffic_record('k_assemble') == dict(bytes=123.0, units=4.0)


def test_shock_workload_shards_by_contiguous_ray_blocks():
    world, rpr = 2, 3
    full = problems.make_shock_problem(bench.CONFIG_ID, n_ray=rpr * world, n_r=16, n_e=4)
    for rank in range(world):
        sl = bench.shard(world, rank, rpr)
        sub = problems.subset_rays(full, sl)
        assert np.array_equal(sub['problem']['u'], full['problem']['u'][sl])
        assert np.array_equal(sub['problem']['eta1'], full['problem']['eta1'][sl])
    assert bench.job_throughput(1000, 2, 4.0) == 1000 * 2 / 4e-3
