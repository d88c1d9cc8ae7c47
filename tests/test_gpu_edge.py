"""Edge and degenerate cases of the GPU path against the oracle: a single level
(the cycle is the coarse solve), a zero right-hand side, meshes with different
cell counts per axis, gamma = 0 (no augmentation), and the size limits."""
import numpy as np
import pytest

from gpu_helpers import context, dev, host, oracle, random_free, rel, sinker

torch = pytest.importorskip("torch")
from paper_2107_00820_gb300 import alstokes as A  # noqa: E402
from oracle.stokes import StokesSolver  # noqa: E402

pytestmark = pytest.mark.gpu


def _coarse_cond(H):
    lv0 = H.levels[0]
    f = np.flatnonzero(lv0.free)
    return np.linalg.cond(lv0.A.toarray()[np.ix_(f, f)])


@pytest.mark.parametrize("d,n", [(2, 8), (3, 4)])
def test_single_level(d, n):
    """levels = 1: no smoothing; the cycle is the dense coarse solve, and FGMRES with
    it matches the oracle's iteration count."""
    pb = sinker(d, n, 1, 1e2, dr=1e4, seed=51)
    ctx = context(pb, rtol=1e-8)
    H = oracle(pb)
    b = random_free(H.levels[-1], 52)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    assert rel(host(x), H.vcycle(b)) <= max(1e-12, 100 * _coarse_cond(H) * 2.2e-16)
    uo, po, its, _ = StokesSolver(H).solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    assert info.converged and info.iterations == its
    assert rel(u, uo) <= 1e-9 and rel(p, po) <= 1e-8


def test_zero_right_hand_side():
    """f = 0 and zero boundary data: no iteration, u = 0 and p = 0 exactly."""
    pb = sinker(2, 16, 3, 1e2, dr=1e4, seed=53)
    ctx = context(pb)
    u, p, info = ctx.solve(np.zeros_like(pb.f), np.zeros_like(pb.u_bc))
    assert info.converged == 1 and info.iterations == 0
    assert not np.any(u) and not np.any(p)


@pytest.mark.parametrize("d,n,levels", [(2, (16, 8), 3), (3, (8, 4, 4), 2)])
def test_anisotropic_mesh(d, n, levels):
    """Different cell counts per axis: cycle parity and an identical solve."""
    pb = sinker(d, n, levels, 1e2, dr=1e4, seed=54)
    ctx = context(pb, sweeps=2, rtol=1e-8)
    H = oracle(pb, steps=2)
    b = random_free(H.levels[-1], 55)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    assert rel(host(x), H.vcycle(b)) <= 1e-11
    uo, po, its, _ = StokesSolver(H).solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    assert info.converged and info.iterations == its
    assert rel(u, uo) <= 1e-9 and rel(p, po) <= 1e-8


def test_gamma_zero():
    """gamma = 0: the plain Stokes system with the same block preconditioner."""
    pb = sinker(2, 16, 3, 0.0, dr=1e2, seed=56)
    ctx = context(pb, rtol=1e-8, maxit=300)
    uo, po, its, _ = StokesSolver(oracle(pb)).solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    assert info.converged and info.iterations == its
    assert rel(u, uo) <= 1e-9 and rel(p, po) <= 1e-8


def test_size_limits_rejected():
    """Meshes whose velocity vector or per-cell staging buffer would need more than
    32-bit indices are refused with ALS_EINVAL before anything is allocated."""
    from paper_2107_00820_gb300 import ALSError, Context
    dummy = [np.zeros(1), np.zeros(1)]
    with pytest.raises(ALSError) as e:
        Context(3, 1024, 2, dummy, 1.0)          # 3 * 2049^3 velocity values > 2^31
    assert e.value.status == A.ALS_EINVAL


def test_profile_samples_one_cycle_in_eight():
    """Kernel timing (als_profile) replays the event-timed graph for one cycle in every 8:
    16 cycles with s = 2 smoothing steps time 2 cycles x 2 s finest-level patch launches,
    and the cycle results do not depend on which graph ran."""
    pb = sinker(3, 8, 2, 1e2, dr=1e4, seed=56)
    ctx = context(pb, sweeps=2, mode=A.ALS_MODE_MIXED)
    H = oracle(pb, steps=2)
    b = dev(random_free(H.levels[-1], 57), torch.float32)
    x0 = torch.zeros_like(b)
    ctx.vcycle(b, x0, A.ALS_PREC_FP32)
    ctx.profile(True)
    outs = []
    for _ in range(16):
        x = torch.zeros_like(b)
        ctx.vcycle(b, x, A.ALS_PREC_FP32)
        outs.append(x)
    torch.cuda.synchronize()
    ms, n = ctx.profile_read()
    ctx.profile(False)
    assert n == 2 * 2 * 2 and ms > 0.0
    for x in outs:
        assert torch.equal(x, x0)


_FUSE_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + '/tests')
from gpu_helpers import context, dev, oracle, random_free, sinker
from paper_2107_00820_gb300 import alstokes as A
pb = sinker(3, 8, 3, 1e2, dr=1e6, seed=58)
ctx = context(pb, mode=A.ALS_MODE_MIXED)
b = dev(random_free(oracle(pb).levels[-1], 59), torch.float32)
x = torch.zeros_like(b)
for _ in range(2):
    ctx.vcycle(b, x, A.ALS_PREC_FP32)
np.save(sys.argv[2], x.cpu().numpy())
"""


def test_fused_patch_gather_bitwise(tmp_path):
    """The FP32 3D cycle forms Z_j inside the cell kernel from the patch outputs; with
    ALS_FUSE_GATHER=0 a separate gather kernel does it.  Same sums in the same order:
    the two cycles must agree bit for bit."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for flag in ("1", "0"):
        path = str(tmp_path / f"x{flag}.npy")
        env = dict(os.environ, ALS_FUSE_GATHER=flag)
        subprocess.run([sys.executable, "-c", _FUSE_SCRIPT, root, path], env=env, check=True, timeout=600)
        outs.append(np.load(path))
    assert np.all(np.isfinite(outs[0]))
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("d,n", [(2, 16), (3, 4)])
def test_smoother_wait_timeout_is_reported_and_recoverable(d, n):
    """ALS_ETIMEOUT: with the poll limit of the FP32 smoother kernel's wait for its
    inverse blocks set to 0, every CTA's first wait gives up at once; the kernel records
    the status, waits (at the default limit) for the bulk copies it had issued, and
    returns.  The call reports ALS_ETIMEOUT, and after the default limit is restored the
    context smooths exactly as before (same bits as a call that never timed out)."""
    pb = sinker(d, n, 2, 1e2, dr=1e3, seed=61)
    ctx = context(pb)
    for lvl in range(1, pb.levels):
        ctx.set_patch_kernel(lvl, 0)             # the TMA-ring variant: the one that waits
    r = dev(np.random.default_rng(62).standard_normal(ctx.nu()), torch.float32)
    z0 = torch.zeros_like(r)
    ctx.star_smooth(1, r, z0, A.ALS_PREC_FP32)
    ctx.set_wait_limit(0)
    with pytest.raises(A.ALSError) as e:
        ctx.star_smooth(1, r, torch.zeros_like(r), A.ALS_PREC_FP32)
    assert e.value.status == A.ALS_ETIMEOUT
    ctx.set_wait_limit(-1)
    z1 = torch.zeros_like(r)
    ctx.star_smooth(1, r, z1, A.ALS_PREC_FP32)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)


def test_mixed_p1_refused_beyond_its_range():
    """Mixed mode with the P1 pairing refuses gamma / mu_min above 0.1 / 2^-24 (the FP32
    cycle's measured limit), naming the pairing that works; P2 and FP64 mode accept the
    same problem."""
    pb = sinker(2, 16, 3, 1e4, dr=1e8, seed=63)      # gamma / mu_min = 1e8
    with pytest.raises(A.ALSError) as e:
        context(pb, mode=A.ALS_MODE_MIXED)
    assert e.value.status == A.ALS_EINVAL and "ALS_SCHUR_P2" in str(e.value)
    context(pb, mode=A.ALS_MODE_MIXED, schur=A.ALS_SCHUR_P2).close()
    context(pb).close()
    ok = sinker(2, 16, 3, 1e2, dr=1e8, seed=63)      # gamma / mu_min = 1e6: within range
    context(ok, mode=A.ALS_MODE_MIXED).close()


def test_solve_history():
    """The residual history: |b| first, one estimate per iteration, the last one the
    info's res_final, falling below rtol |b| at the end."""
    pb = sinker(2, 16, 3, 1e2, dr=1e4, seed=64)
    ctx = context(pb, rtol=1e-8)
    _, _, info = ctx.solve(pb.f, pb.u_bc)
    h = ctx.solve_history()
    assert len(h) == info.iterations + 1
    assert h[0] == info.res0 and h[-1] == info.res_final
    assert h[-1] <= 1e-8 * h[0] < h[-2]


def test_null_vectors_refused_through_the_abi():
    """Every per-level entry point refuses a NULL vector with ALS_EINVAL before it queues
    any work, and the context stays usable: an apply after the refusals matches the
    oracle."""
    pb = sinker(2, 8, 2, 1e2, dr=1e3, seed=65)
    ctx = context(pb)
    lib, c = ctx._lib, ctx._ctx
    v = torch.zeros(ctx.nu(), dtype=torch.float64, device="cuda")
    p = A.c_void_p(v.data_ptr())
    calls = [("als_apply_agamma", (c, 1, 0, None, p)), ("als_vcycle", (c, 0, p, None)),
             ("als_star_smooth", (c, 1, 0, None, p)), ("als_star_smooth", (c, 1, 0, p, None)),
             ("als_prolong", (c, 1, 0, None, p)), ("als_prolong", (c, 1, 0, p, None)),
             ("als_restrict", (c, 1, 0, None, p)), ("als_restrict", (c, 1, 0, p, None)),
             ("als_coarse_solve", (c, 0, None, p)), ("als_coarse_solve", (c, 0, p, None)),
             ("als_apply_stokes", (c, p, None, p, p)), ("als_patch_inverse", (c, 1, 0, None)),
             ("als_load_patch_inverses", (c, 1, None)), ("als_load_coarse_inverse", (c, None))]
    for name, args in calls:
        assert getattr(lib, name)(*args) == A.ALS_EINVAL, name
        assert lib.als_last_error(c)
    H = oracle(pb)
    x = random_free(H.levels[-1], 66)
    y = torch.zeros_like(v)
    ctx.apply_agamma(dev(x), y)
    assert rel(host(y), H.levels[-1].A @ x) <= 1e-12


_SPLIT_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + '/tests')
from gpu_helpers import context, dev, host, oracle, random_free, rel, sinker
from paper_2107_00820_gb300 import alstokes as A
out = []
for d, n, L in ((2, 16, 3), (3, 8, 3)):
    pb = sinker(d, n, L, 1e2, dr=1e3, seed=81)
    H = oracle(pb, steps=2)
    ctx = context(pb, sweeps=2, mode=A.ALS_MODE_MIXED)
    lv = H.levels[-1]
    r = random_free(lv, 82)
    z = torch.zeros(lv.mesh.nu, dtype=torch.float32, device="cuda")
    ctx.star_smooth(L - 1, dev(r, torch.float32), z, A.ALS_PREC_FP32)
    out.append(rel(host(z), H.patches[L - 1].apply(r)))
    b = random_free(lv, 83)
    x = torch.zeros(lv.mesh.nu, dtype=torch.float32, device="cuda")
    ctx.vcycle(dev(b, torch.float32), x, A.ALS_PREC_FP32)
    out.append(rel(host(x), H.vcycle(b)))
    for variant in (0, 2):
        for lvl in range(1, L):
            ctx.set_patch_kernel(lvl, variant)
        x = torch.zeros(lv.mesh.nu, dtype=torch.float32, device="cuda")
        ctx.vcycle(dev(b, torch.float32), x, A.ALS_PREC_FP32)
        out.append(rel(host(x), H.vcycle(b)))
print(" ".join(f"{v:.3e}" for v in out))
"""


@pytest.mark.parametrize("flag", ["1", "0"])
def test_split_and_whole_star_storage(flag):
    """FP32 star storage split (interior stars block-packed, boundary stars restricted to
    their free dofs and applied by their own kernel) and whole (every star padded): the
    smoother and the FP32 cycle (TMA-ring and direct-load variants) match the oracle
    within FP32 rounding either way, in 2D and 3D, on meshes small enough that the
    default would store them whole."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, ALS_SPLIT_STARS=flag)
    r = subprocess.run([sys.executable, "-c", _SPLIT_SCRIPT, root], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    errs = [float(v) for v in r.stdout.split()]
    assert len(errs) == 8 and all(e <= 1e-4 for e in errs), errs
