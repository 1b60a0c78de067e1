"""The general product C = X^t Y (ata_gemm_tn, the HASA step of Section
4.2.2 as an entry point) on the GPU against the oracle, through the C ABI.

Tolerances: FP64 and the FP64 emulation componentwise
max |C - C_ref| / (|X|^t |Y|) <= 1e-11, and bf16x3 normwise
||C - C_ref||_F / ||C_ref||_F <= 1e-6, as for A^t A.  TF32 rounds every
operand to 11 significant bits (unit u = 2^-11) and accumulates in FP32.  For
A^t A the norm is dominated by the diagonal, whose rounding errors average
out, hence its 1e-3; a product of two independent operands keeps an error of
about u relative in every entry, and each Strassen level (operand sums, four
products combined) roughly doubles it.  The general-product test therefore
holds TF32 to normwise 4u = 2^-9 at two Strassen levels.  Strassen bounds
are normwise only, so inputs with scaled columns are measured normwise.
Winograd's variant has the larger error constant (18 against Strassen's 12
per level in the normwise bound, Higham, Accuracy and Stability of Numerical
Algorithms, Thms. 23.2-23.3), so its normwise bounds are 1.5x per level
looser.  Exact-integer inputs match bitwise in every mode.
"""
import numpy as np
import pytest

import oracle
import paper_1902_02104_gb300 as ata
from paper_1902_02104_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL = [ata.ATA_F64, ata.ATA_F32_BF16X3, ata.ATA_F32_TF32, ata.ATA_F64_OZAKI]


def in_dtype(dtype):
    return np.float64 if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI) else np.float32


def run(X_np, Y_np, dtype, cutoff, **opts):
    import torch
    m, p = X_np.shape
    r = Y_np.shape[1]
    plan = ata.GemmPlan(m, p, r, dtype, cutoff, **opts)
    X = torch.from_numpy(np.ascontiguousarray(X_np)).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(Y_np)).cuda()
    C = plan(X, Y)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return C.cpu().numpy(), plan


def normwise(C, R):
    return float(np.linalg.norm(C - R) / max(np.linalg.norm(R), 1e-300))


def componentwise(C, R, G):
    d = np.abs(C - R)
    zero = G == 0
    assert np.all(d[zero] == 0)
    return float(np.max(d[~zero] / G[~zero])) if np.any(~zero) else 0.0


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("m,p,r,cutoff,fuse", [(512, 384, 300, 64, 0), (700, 333, 517, 64, 1), (300, 129, 1000, 32, 0),
                                               (1030, 260, 260, 128, 1), (100, 1, 7, 16, 0)])
def test_gemm_exact_integers_bitwise(gpu, dtype, m, p, r, cutoff, fuse):
    if dtype != ata.ATA_F64 and cutoff < 64:
        cutoff = 64
    dt = in_dtype(dtype)
    X = inputs.integers(m, p, seed=m + p).astype(dt)
    Y = inputs.integers(m, r, seed=m + r + 7).astype(dt)
    C, plan = run(X, Y, dtype, cutoff, fuse_levels=fuse)
    assert np.array_equal(C, oracle.gemm_tn(X, Y)), plan.info


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("variant", [ata.ATA_STRASSEN, ata.ATA_WINOGRAD])
def test_gemm_float_tolerance(gpu, dtype, variant):
    m, p, r = 1500, 900, 700
    if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI):
        X, Y = inputs.normal(m, p, seed=1), inputs.normal(m, r, seed=2)
    else:
        X, Y = inputs.scaled_cols(m, p, seed=1), inputs.scaled_cols(m, r, seed=2)
    C, plan = run(X, Y, dtype, 256, variant=variant)
    assert plan.info["max_strassen_levels"] >= 1
    ref = oracle.gemm_tn(X, Y)
    if dtype in (ata.ATA_F64, ata.ATA_F64_OZAKI):
        err = componentwise(C, ref, oracle.gemm_tn(X, Y, absval=True))
        assert err <= 1e-11, err
    else:
        levels = plan.info["max_strassen_levels"]
        assert levels <= 2
        growth = 1.5 ** levels if variant == ata.ATA_WINOGRAD else 1.0
        err = normwise(C, ref)
        assert err <= (1e-6 if dtype == ata.ATA_F32_BF16X3 else 2.0 ** -9) * growth, err


@pytest.mark.parametrize("dtype", [ata.ATA_F64, ata.ATA_F32_BF16X3])
def test_gemm_leading_dimensions_and_repointing(gpu, dtype):
    import torch
    m, p, r = 400, 250, 190
    dt = in_dtype(dtype)
    Xb = inputs.integers(m, p + 13, seed=3).astype(dt)
    Yb = inputs.integers(m, r + 5, seed=4).astype(dt)
    plan = ata.GemmPlan(m, p, r, dtype, 64)
    X = torch.from_numpy(Xb).cuda()[:, 3:3 + p]
    Y = torch.from_numpy(Yb).cuda()[:, 1:1 + r]
    Cbig = torch.full((p, r + 9), 7.0, dtype=torch.float64, device="cuda")
    C = Cbig[:, 2:2 + r]
    plan(X, Y, C)
    torch.cuda.synchronize()
    want = oracle.gemm_tn(Xb[:, 3:3 + p], Yb[:, 1:1 + r])
    assert np.array_equal(C.cpu().numpy(), want)
    # columns outside the window untouched
    assert torch.all(Cbig[:, :2] == 7.0) and torch.all(Cbig[:, 2 + r:] == 7.0)
    # dense operands on the same plan (tables rebuilt for the new leading dimensions)
    X2 = torch.from_numpy(np.ascontiguousarray(Xb[:, 3:3 + p])).cuda()
    Y2 = torch.from_numpy(np.ascontiguousarray(Yb[:, 1:1 + r])).cuda()
    C2 = plan(X2, Y2)
    torch.cuda.synchronize()
    assert np.array_equal(C2.cpu().numpy(), want)


@pytest.mark.parametrize("dtype", ALL)
def test_gemm_degenerate_shapes(gpu, dtype):
    import torch
    dt = in_dtype(dtype)
    # m = 0: C = 0
    C, _ = run(np.zeros((0, 70), dt), np.zeros((0, 50), dt), dtype, 64)
    assert C.shape == (70, 50) and np.all(C == 0)
    # p = 0 or r = 0: nothing to write
    plan = ata.GemmPlan(10, 0, 5, dtype, 64)
    out = plan(torch.zeros((10, 0), dtype=torch.float64 if dt == np.float64 else torch.float32, device="cuda"),
               torch.zeros((10, 5), dtype=torch.float64 if dt == np.float64 else torch.float32, device="cuda"))
    assert tuple(out.shape) == (0, 5)


def test_gemm_plan_rejects_ata_entry_points(gpu):
    import torch
    plan = ata.GemmPlan(64, 32, 16, ata.ATA_F64, 16)
    A = torch.zeros((64, 32), dtype=torch.float64, device="cuda")
    C = torch.zeros(32 * 33 // 2, dtype=torch.float64, device="cuda")
    lib = ata.load()
    st = lib.ata_execute(plan.handle, ata.ctypes.c_void_p(A.data_ptr()), 32, ata.ctypes.c_void_p(C.data_ptr()), None)
    assert st == ata.ATA_EINVAL
    ata_plan = ata.Plan(64, 32, ata.ATA_F64, 16)
    st = lib.ata_gemm_tn(ata_plan.handle, ata.ctypes.c_void_p(A.data_ptr()), 32, ata.ctypes.c_void_p(A.data_ptr()), 32,
                         ata.ctypes.c_void_p(C.data_ptr()), 32, None)
    assert st == ata.ATA_EINVAL


def test_gemm_deterministic_and_ozaki_sampled_large(gpu):
    # the top C_12 product of a 10000^2 A^t A: X, Y = 10000 x 5000
    import torch
    m, p, r = 10000, 5000, 5000
    X = inputs.normal(m, p, seed=11)
    Y = inputs.normal(m, r, seed=12)
    plan = ata.GemmPlan(m, p, r, ata.ATA_F64_OZAKI, 0)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    C1 = plan(Xd, Yd)
    C2 = plan(Xd, Yd)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    assert torch.equal(C1, C2)
    rng = np.random.default_rng(5)
    I = rng.integers(0, p, 1500)
    J = rng.integers(0, r, 1500)
    got = C1.cpu().numpy()[I, J]
    want = oracle.gemm_entries(X, Y, I, J)
    G = oracle.gemm_entries(X, Y, I, J, absval=True)
    assert float(np.max(np.abs(got - want) / G)) <= 1e-11
