"""The allocation-free residual-norm entry point against the existing path.

amg_residual_norm_noalloc serves callers that cannot allocate device memory
when they need the check (a device heap owned by another framework's pool, a
frozen memory budget, a monitor that must not disturb the application's
allocator).  It must agree with the allocating path -- amg_spmv followed by
the norms -- on consecutive calls that share its fixed scratch array.
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_residual_norm_matches_spmv_path(gen):
    torch = pytest.importorskip("torch")
    from paper_1410_2153_gb300 import asmg
    assert torch.cuda.is_available()
    m = gen.grid2d(97, 3, graded=True)        # 9,025 free dofs: several blocks and a ragged tail
    s = asmg.Solver(m)
    free = m.bflag == 0
    rng = np.random.default_rng(17)
    for trial in range(3):                     # consecutive calls share the scratch
        b = rng.uniform(-1, 1, m.nv) * (trial + 1)
        u = rng.uniform(-1, 1, m.nv)
        db, du = torch.from_numpy(b).cuda(), torch.from_numpy(u).cuda()
        torch.cuda.synchronize()
        rn, bn = asmg.amg_residual_norm_noalloc(s.h, db, du)
        y = s.spmv(du).cpu().numpy()           # existing entry point
        ref_r = np.linalg.norm((b - y)[free])
        ref_b = np.linalg.norm(b[free])
        assert abs(rn - ref_r) <= 1e-12 * ref_r, (trial, rn, ref_r)
        assert abs(bn - ref_b) <= 1e-12 * ref_b, (trial, bn, ref_b)
    # a warm call creates no device memory: the driver's free-memory count
    # is the same before and after several more calls
    db, du = torch.from_numpy(b).cuda(), torch.from_numpy(u).cuda()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        asmg.amg_residual_norm_noalloc(s.h, db, du)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    # host arrays are refused rather than staged through new memory
    with pytest.raises(asmg.AsmgError) as e:
        asmg.amg_residual_norm_noalloc(s.h, np.zeros(m.nv), np.zeros(m.nv))
    assert e.value.code == asmg.ASMG_ERR_INVALID_ARG
    s.close()
