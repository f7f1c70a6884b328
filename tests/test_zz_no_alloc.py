"""The allocation-free electron count agrees with the regular entry point.

marnoldi_count_noalloc is for callers that cannot allocate device memory
(code under another framework's memory manager, or a request path that must
not allocate): its reduction scratch is a fixed array inside the library.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""

import numpy as np
import pytest

from tbsynth import config_c1

pytestmark = pytest.mark.gpu

KT = 0.1


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_3218_gb300 as mm
    from paper_1307_3218_gb300 import build as b
    b.build()
    mm.load()
    return mm


def test_count_noalloc_matches_solve_twice(m):
    import torch
    t = config_c1(seed=0)
    for mu in (1.7, -3.25):
        ctx = m.setup_system(t, m.MARNOLDI_FP64)
        m.marnoldi_solve(ctx, None, 30, 0, 0.0, KT, mu)
        E_ref, _, N_ref = m.marnoldi_energy(ctx)
        nue, eps, w = m.marnoldi_column_stats(ctx)
        m.marnoldi_destroy(ctx)
        eps_d = torch.tensor(eps, dtype=torch.float64, device="cuda")
        w_d = torch.tensor(w, dtype=torch.float64, device="cuda")
        nue_d = torch.tensor(nue, dtype=torch.int32, device="cuda")
        out = torch.empty(2, dtype=torch.float64, device="cuda")
        for _ in range(2):                      # two calls in a row share the scratch
            out.fill_(float("nan"))
            m.marnoldi_count_noalloc(eps_d, w_d, nue_d, eps.shape[0], eps.shape[1], mu, KT, out)
            torch.cuda.synchronize()
            N, E = out.cpu().numpy()
            assert N == pytest.approx(N_ref, rel=1e-10)
            assert E == pytest.approx(E_ref, rel=1e-10)
        # NULL nu_eff: every level counts (padding levels carry w = 0)
        m.marnoldi_count_noalloc(eps_d, w_d, None, eps.shape[0], eps.shape[1], mu, KT, out)
        torch.cuda.synchronize()
        assert out[0].item() == pytest.approx(N_ref, rel=1e-10)


def test_count_noalloc_rejects_oversize(m):
    import torch
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(m.MarnoldiError) as ei:
        m.marnoldi_count_noalloc(x, x, None, 16_777_217, 1, 0.0, KT, x)
    assert ei.value.code == m.marnoldi.MARNOLDI_EINVAL
    assert "16777216" in str(ei.value)


def test_count_noalloc_allocates_nothing(m):
    """After a first call (which loads the library's device code on this device), further calls
    leave the device's free memory and torch's allocated bytes unchanged."""
    import torch
    n, nu = 4096, 30
    g = torch.Generator(device="cpu").manual_seed(3)
    eps = torch.randn(n * nu, generator=g, dtype=torch.float64).cuda()
    w = torch.rand(n * nu, generator=g, dtype=torch.float64).cuda()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    m.marnoldi_count_noalloc(eps, w, None, n, nu, 0.0, KT, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for q in range(5):
        m.marnoldi_count_noalloc(eps, w, None, n, nu, 0.1 * q, KT, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0
    assert torch.cuda.memory_allocated() == alloc0


def test_count_noalloc_binding_checks_tensors(m):
    import torch
    good = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for bad in (torch.zeros(64, dtype=torch.float32, device="cuda"),     # dtype
                torch.zeros(63, dtype=torch.float64, device="cuda"),     # too short for 8 x 8
                torch.zeros(128, dtype=torch.float64, device="cuda")[::2]):  # strided
        with pytest.raises(m.MarnoldiError) as ei:
            m.marnoldi_count_noalloc(bad, good, None, 8, 8, 0.0, KT, out)
        assert ei.value.code == m.marnoldi.MARNOLDI_EINVAL
    with pytest.raises(m.MarnoldiError) as ei:
        m.marnoldi_count_noalloc(good, good, torch.zeros(8, dtype=torch.int64, device="cuda"),
                                 8, 8, 0.0, KT, out)
    assert ei.value.code == m.marnoldi.MARNOLDI_EINVAL
