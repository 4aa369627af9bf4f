"""pfc_advect_v_static, the allocation-free velocity pass (its per-cell
scratch is a static device array of the library), against pfc_advect_v
(scratch in the caller's workspace), both through the C ABI on the same
seeded state. Two calls in a row must agree, so the shared static array
carries nothing from one call to the next; a state split into two cell
ranges must agree with the whole; an oversized call is refused.

Tolerance: both paths run the same kernels on the same inputs, so the
results agree to the last bit in practice; the bound allows a few ulps
(1e-13 relative to max|f| in FP64, 1e-6 in FP32) and the moments within the
same fraction of their absolute scale.
"""
import numpy as np
import pytest

from paper_2109_06743_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2109_06743_gb300 import build
    build.build()
    return torch


def _setup(precision, nv, nx=6, ny=5, seed=11, nshear=5):
    from gpu_util import AbiRunner
    cfg = W.harris(nx=nx, ny=ny, nv=nv, lx=25.6 * nx / 128, ly=12.8 * ny / 64, precision=precision)
    cfg.nshear = nshear
    V = nv ** 3
    f0 = [W.random_blocks((cfg.ncell, V), seed + k) ** 4 for k in range(len(cfg.species))]
    if precision == 32:
        f0 = [f.astype(np.float32).astype(np.float64) for f in f0]
    eb = W.random_fields(cfg.ncell, seed + 7, e_scale=0.5, b_scale=1.0)
    eb[0, 3:] = 0.0  # a cell without magnetic field
    return cfg, AbiRunner(cfg, f0, eb=eb)


def _close(a, b, precision, scale):
    """|a - b| <= rel * scale elementwise (scale broadcasts)."""
    tol = (1e-13 if precision == 64 else 1e-6) * np.broadcast_to(scale, a.shape)
    ratio = float((np.abs(a - b) / tol).max())
    assert ratio <= 1.0, ratio


@pytest.mark.parametrize("precision,nv,nshear", [(64, 8, 5), (32, 12, 5), (32, 8, 3)])
def test_static_scratch_matches_workspace_pass(gpu, precision, nv, nshear):
    from paper_2109_06743_gb300 import abi
    torch = gpu
    cfg, r = _setup(precision, nv, nshear=nshear)
    for s in range(len(cfg.species)):
        f_b = r.f[s].clone()
        start = f_b.clone()
        for dt in (0.02, -0.013):  # two calls in a row
            m_a, m_b = r.mom(), r.mom()
            abi.pfc_advect_v(r.ctx, s, dt, m_a, stream=r.stream)
            abi.pfc_advect_v_static(r.desc, s, f_b, r.eb, cfg.ncell, dt, m_b, stream=r.stream)
            torch.cuda.synchronize()
            fa = r.f[s].double().cpu().numpy()
            fb = f_b.double().cpu().numpy()
            _close(fa, fb, precision, fa.max())
            ma, mb = m_a.cpu().numpy(), m_b.cpu().numpy()
            _close(ma, mb, precision, np.abs(ma).max(axis=0, keepdims=True) + 1e-300)
        assert not torch.equal(start, f_b)  # the pass did move f
    r.close()


def test_static_scratch_split_ranges_and_limit(gpu):
    from paper_2109_06743_gb300 import abi
    torch = gpu
    cfg, r = _setup(32, 8, nx=7, ny=4, seed=23)
    s, dt = 1, 0.03
    f_b = r.f[s].clone()
    m_a, m_b = r.mom(), r.mom()
    abi.pfc_advect_v(r.ctx, s, dt, m_a, stream=r.stream)
    k = cfg.ncell // 3
    es = f_b.element_size()
    V = f_b.shape[1]
    abi.pfc_advect_v_static(r.desc, s, f_b, r.eb, k, dt, m_b, stream=r.stream)
    abi.pfc_advect_v_static(r.desc, s, f_b.data_ptr() + k * V * es, r.eb.data_ptr() + k * 6 * 8, cfg.ncell - k, dt,
                            m_b.data_ptr() + k * 20 * 8, stream=r.stream)
    torch.cuda.synchronize()
    fa = r.f[s].double().cpu().numpy()
    _close(fa, f_b.double().cpu().numpy(), 32, fa.max())
    ma = m_a.cpu().numpy()
    _close(ma, m_b.cpu().numpy(), 32, np.abs(ma).max(axis=0, keepdims=True) + 1e-300)
    # beyond the static scratch: refused before any launch, state untouched
    before = f_b.clone()
    with pytest.raises(abi.VlasovError) as e:
        abi.pfc_advect_v_static(r.desc, s, f_b, r.eb, abi.STATIC_SCRATCH_CELLS + 1, dt, None, stream=r.stream)
    assert e.value.status == abi.VL_EINVAL and "split the call" in str(e.value)
    torch.cuda.synchronize()
    assert torch.equal(before, f_b)
    # an empty range is a no-op
    abi.pfc_advect_v_static(r.desc, s, f_b, r.eb, 0, dt, None, stream=r.stream)
    r.close()


def test_static_scratch_1d1v_matches_workspace_pass(gpu):
    """The 1D1V branch of the allocation-free pass (one thread per spatial
    cell, E read at stride 6) against pfc_advect_v on the Landau set-up,
    two calls in a row."""
    from gpu_util import AbiRunner
    from paper_2109_06743_gb300 import abi
    torch = gpu
    cfg = W.landau()
    f0 = W.landau_state(cfg)
    eb = np.zeros((cfg.ncell, 6))
    eb[:, 0] = 0.3 * np.sin(np.linspace(0.0, 2.0 * np.pi, cfg.ncell, endpoint=False))
    eb[:, 1:] = 7.0  # other components must not be read
    r = AbiRunner(cfg, f0, eb=eb)
    f_b = r.f[0].clone()
    for dt in (0.05, -0.03):
        m_a, m_b = r.mom(), r.mom()
        abi.pfc_advect_v(r.ctx, 0, dt, m_a, stream=r.stream)
        abi.pfc_advect_v_static(r.desc, 0, f_b, r.eb, cfg.ncell, dt, m_b, stream=r.stream)
        torch.cuda.synchronize()
        fa = r.f[0].cpu().numpy()
        _close(fa, f_b.cpu().numpy(), 64, fa.max())
        ma = m_a.cpu().numpy()
        _close(ma, m_b.cpu().numpy(), 64, np.abs(ma).max(axis=0, keepdims=True) + 1e-300)
    r.close()


def test_static_scratch_full_array(gpu):
    """One FP32 8^3 call over exactly VL_STATIC_SCRATCH_CELLS cells (the whole
    static array, 67 MB of f) against the workspace pass of the same cells."""
    from gpu_util import AbiRunner
    from paper_2109_06743_gb300 import abi
    torch = gpu
    n = abi.STATIC_SCRATCH_CELLS
    cfg = W.harris(nx=256, ny=n // 256, nv=8, lx=25.6 * 2, ly=12.8 * (n // 256) / 64, precision=32)
    assert cfg.ncell == n
    V = 8 ** 3
    f0 = [W.random_blocks((n, V), 31 + k, dtype=np.float32) ** 4 for k in range(2)]
    eb = W.random_fields(n, 37, e_scale=0.5, b_scale=1.0)
    r = AbiRunner(cfg, f0, eb=eb)
    s = 0
    f_b = r.f[s].clone()
    m_a, m_b = r.mom(), r.mom()
    abi.pfc_advect_v(r.ctx, s, 0.02, m_a, stream=r.stream)
    abi.pfc_advect_v_static(r.desc, s, f_b, r.eb, n, 0.02, m_b, stream=r.stream)
    torch.cuda.synchronize()
    fa = r.f[s].double().cpu().numpy()
    _close(fa, f_b.double().cpu().numpy(), 32, fa.max())
    ma = m_a.cpu().numpy()
    _close(ma, m_b.cpu().numpy(), 32, np.abs(ma).max(axis=0, keepdims=True) + 1e-300)
    r.close()
