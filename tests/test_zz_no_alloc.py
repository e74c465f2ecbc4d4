"""mlmc_level_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (a framework that owns all device memory and passes the library
only its own buffers, or a serving loop that forbids allocation after start-up)
get a context-free entry point whose scratch lives in a static device array.
This test checks, through the C ABI, that two calls in a row give the same
results as the context-based mlmc_level_solve, and that a batch beyond the
array's capacity is refused with a clear error.  It is collected last and needs
nothing from earlier tests.
"""
import numpy as np
import pytest

from gpu_common import device, lib, to_dev, torch
from inputs import smooth_lognormal_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    device()
    return lib()


def _reference(M, n, af, a_prec, prec, delta, qoi, box):
    kw = dict(n0=n, m=2, L_max=0, kind=0, K=4, sigma2=1.0, corr_len=0.3, seed=0, qoi=qoi)
    if box is not None:
        kw["box"] = box
    h = M.mlmc_create(M.make_problem(**kw), 0)
    try:
        M.mlmc_set_precond(h, M.MLMC_PC_JACOBI)    # the allocation-free entry point runs Jacobi-PCG
        S = af.shape[0]
        dt = torch.float64 if a_prec == M.MLMC_FP64 else torch.float32
        Q = torch.empty(S, dtype=torch.float64, device=device())
        rr = torch.empty(S, dtype=torch.float64, device=device())
        fl = torch.empty(S, dtype=torch.int32, device=device())
        M.mlmc_level_solve(h, n, S, to_dev(af, dt), a_prec, n, prec, M.MLMC_CG, delta, 100000, None, Q, None, rr, fl)
        torch.cuda.synchronize()
        return Q.cpu().numpy(), rr.cpu().numpy(), fl.cpu().numpy()
    finally:
        M.mlmc_destroy(h)


def _noalloc(M, n, af, a_prec, prec, delta, qoi, box):
    S = af.shape[0]
    dt = torch.float64 if a_prec == M.MLMC_FP64 else torch.float32
    a = to_dev(af, dt)
    Q = torch.empty(S, dtype=torch.float64, device=device())
    it = torch.empty(S, dtype=torch.int32, device=device())
    rr = torch.empty(S, dtype=torch.float64, device=device())
    fl = torch.empty(S, dtype=torch.int32, device=device())
    M.mlmc_level_solve_noalloc(0, n, S, a, a_prec, n, prec, delta, 100000, qoi, box, 1.0, Q, it, rr, fl)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), rr.cpu().numpy(), fl.cpu().numpy()


def test_noalloc_matches_level_solve_on_two_calls_in_a_row(M):
    cases = [
        # n, S, master precision, inner precision, delta, qoi, box
        (64, 7, M.MLMC_FP64, M.MLMC_FP64, 1e-11, 0, None),
        (32, 13, M.MLMC_FP32, M.MLMC_FP16S, 1e-6, 1, (0.25, 0.75, 0.25, 0.75)),
        # n = 128: one 512-thread CTA per system (the large-system class), BF16-stored coefficient
        (128, 8, M.MLMC_FP32, M.MLMC_BF16S, 1e-6, 0, None),
    ]
    for i, (n, S, ap, prec, delta, qoi, box) in enumerate(cases):
        af = smooth_lognormal_field(n, S, seed=100 + i, log_sd=1.0)
        Qr, rrr, flr = _reference(M, n, af, ap, prec, delta, qoi, box)
        Qn, rrn, fln = _noalloc(M, n, af, ap, prec, delta, qoi, box)
        assert np.all(flr == M.MLMC_F_CONVERGED) and np.all(fln == M.MLMC_F_CONVERGED)
        assert np.all(rrn < delta)
        # same kernel and fixed-order reductions: the parity tolerance of the FP64 tests
        assert np.allclose(Qn, Qr, rtol=1e-12, atol=0)
        assert np.allclose(rrn, rrr, rtol=1e-9, atol=1e-18)


def test_noalloc_rejects_batches_beyond_its_scratch(M):
    n, S = 256, 100   # about 330 MB of FP64 scratch
    a = torch.ones((S, (n + 1) ** 2), dtype=torch.float64, device=device())
    Q = torch.empty(S, dtype=torch.float64, device=device())
    with pytest.raises(M.MlmcError) as ei:
        M.mlmc_level_solve_noalloc(0, n, S, a, M.MLMC_FP64, n, M.MLMC_FP64, 1e-8, 1000, 0, None, 1.0, Q)
    assert ei.value.status == M.MLMC_E_ARG
    assert "MLMC_NOALLOC_SCRATCH_BYTES" in M.mlmc_last_error(None)


@pytest.mark.parametrize("box", [(0.25, 0.2, 0.25, 0.75), (0.25, 0.75, -0.25, 0.75), (0.25, 0.75, 0.25, 1.5),
                                 (0.25, float("nan"), 0.25, 0.75), (0.3, 0.75, 0.25, 0.75)])
def test_noalloc_rejects_bad_qoi_boxes(M, box):
    # inverted, outside the unit square, not finite, or off the grid lines of n = 16 (0.3 * 16 = 4.8)
    n, S = 16, 2
    a = torch.ones((S, (n + 1) ** 2), dtype=torch.float64, device=device())
    Q = torch.empty(S, dtype=torch.float64, device=device())
    with pytest.raises(M.MlmcError) as ei:
        M.mlmc_level_solve_noalloc(0, n, S, a, M.MLMC_FP64, n, M.MLMC_FP64, 1e-8, 1000, 1, box, 1.0, Q)
    assert ei.value.status == M.MLMC_E_ARG
    assert "box" in M.mlmc_last_error(None)
