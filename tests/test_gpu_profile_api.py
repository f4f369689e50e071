"""GPU tests of the timing and progress entry points (fth_profile_enable / _read,
fth_pool_profile, fth_pool_progress)."""
import numpy as np
import pytest

import fth_synth as syn

from gpu_util import gpu_ready

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_ready(), reason="needs a CUDA GPU and libfth.so")]


def test_context_profile_times_each_kernel_class_and_resets_on_read():
    from paper_1402_2095_gb300 import FTH
    M, _, _ = syn.dense_spd(256, 1.0, 100.0, seed=3)
    a, c = syn.random_gle(4, seed=5, rate=3.0)
    f = FTH(M=M.astype(np.float32), a_p=a, c_p=c, dt=0.01, replicas=64, seed=1,
            precision="tf32", track="diag", block=10)
    f.run(3)
    f.profile(True)
    f.run(20)
    prof = f.profile_read()
    f.profile(False)
    assert prof["force_tc"][1] >= 20 and prof["gle_dense"][1] >= 20
    assert all(ms > 0.0 for ms, _ in prof.values())
    assert f.profile_read() == {}          # counts are since the last read
    f.close()


def test_pool_profile_and_progress():
    from paper_1402_2095_gb300 import Pool
    M, _, _ = syn.dense_spd(200, 1.0, 100.0, seed=4)
    a, c = syn.random_gle(4, seed=6, rate=3.0)
    pool = Pool(1 << 26, replicas=32, max_problems=4)
    h = pool.add(M, a_p=a, c_p=c, dt=0.01, seed=2, block=5, pairs=syn.diag_pairs(200)[:8])
    pool.run(30)
    prof = pool.profile(10)
    for k in ("pool_force", "pool_gle", "pool_accum"):
        assert prof[k][1] >= 10 and prof[k][0] > 0.0, k
    rel, blocks = pool.progress()
    assert blocks[h] >= 2 and np.isfinite(rel[h]) and rel[h] > 0.0
    assert all(np.isnan(rel[k]) for k in range(len(rel)) if k != h)
    pool.close()
