"""GPU parity: every kernel of the CUDA path, called through the C ABI, against
the FP64 CPU oracle on the same seeded inputs.

Tolerances: FP64 kernels agree to 1e-12 relative; FP32 smoothing agrees to
the FP32 round-off level (2e-6 relative, about 30 units of FP32 rounding:
each node update sums some 60 products); the mixed solve reaches the same
1e-10 relative residual and its error against the FP64 oracle solution is
bounded and reported.  Every comparison is both norm-wise and element-wise:
``rel`` is the larger of |a - b|_2 / |b|_2 and max|a - b| / max|b|, so a
localised error (a wall row, a strip seam) cannot hide under a norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_1904_03808_gb300 import MG_FP64, MG_MIXED, Context, inputs as I, make_state  # noqa: E402

MU = I.TABLE1["mu"]
K = I.TABLE1["K"]
LAM = I.lame_lambda(K, MU)
TOL64 = 1e-12


def g(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def c(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    """max(|a - b|_2 / |b|_2, max|a - b| / max|b|)."""
    d = (np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return max(np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300),
               np.abs(d).max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300))


SHAPES = [(8, 8, 8), (16, 16, 16), (24, 16, 8), (16, 8, 12), (8, 12, 6), (32, 32, 32)]


def ctx_for(shape, precision=MG_FP64, w=None, **kw):
    nx, ny, nz = shape
    h = 2e-2 / nx
    bc = stz = None
    if w is not None:
        bc, stz, h = w.bc_values(), w.stz, w.h
    return Context(nx, ny, nz, h, K, MU, bc=bc, stz=stz, precision=precision, **kw)


def rand_corner(rng, shape, walls=True):
    nx, ny, nz = shape
    x = rng.uniform(-1, 1, size=(3, nz + 1, ny, nx))
    if not walls:
        x[:, 0] = 0
        x[:, nz] = 0
    return x


@pytest.mark.parametrize("shape", SHAPES)
def test_hierarchy_and_galerkin_tables(shape):
    ctx = ctx_for(shape)
    mg = O.MG(*shape, LAM, MU)
    assert ctx.levels == mg.levels
    for l in range(mg.levels):
        assert ctx.level_dims(l) == mg.dims(l)
        S_gpu, S_ora = ctx.level_stencil(l), mg.stencil(l)
        assert np.allclose(S_gpu, S_ora, rtol=0, atol=1e-14 * np.abs(S_ora).max())


@pytest.mark.parametrize("shape", [(64, 32, 32), (256, 32, 32), (128, 40, 32), (72, 40, 16),
                                   (16, 8, 12), (512, 32, 32), (192, 24, 16), (384, 32, 32),
                                   (768, 64, 64)])
def test_residual32_every_level(shape):
    """FP32 residual of the mixed-precision V-cycles against the oracle's on
    the same (FP32-rounded) arrays: the persistent row-strip kernel on the
    finest level for rows of 64/128/192/256 nodes with at least 9 rows (ragged
    strips at ny = 40), one thread per node otherwise, coarse levels."""
    rng = np.random.default_rng(11)
    ctx = ctx_for(shape, precision=MG_MIXED)
    mg = O.MG(*shape, LAM, MU)
    for l in range(max(mg.levels - 1, 1)):
        d = mg.dims(l)
        x = rand_corner(rng, d).astype(np.float32).astype(np.float64)
        b = rand_corner(rng, d).astype(np.float32).astype(np.float64)
        if l > 0:
            x[:, [0, d[2]]] = 0
        r = torch.full(x.shape, float("nan"), device="cuda", dtype=torch.float32)
        ctx.residual32(l, g(b, torch.float32), g(x, torch.float32), r)
        want = O.residual(mg.stencil(l), b, x)
        got = c(r).astype(np.float64)
        assert np.isfinite(got).all()
        assert rel(got, want) <= 1e-6, (l, rel(got, want))
    ctx.close()


@pytest.mark.parametrize("shape", [(256, 32, 32), (128, 40, 32), (192, 24, 16), (64, 64, 64),
                                   (128, 64, 32), (72, 40, 16), (16, 8, 12)])
def test_residual_restrict32(shape):
    """The FP32 residual and its restriction as the V-cycle computes them:
    fused without storing the residual on the finest level where the row-strip
    kernel takes the grid (rows of 64/128/192/256 nodes; ny = 40 leaves a
    ragged last strip of 4 rows), else residual then restriction; against the oracle's restriction of its residual on the same
    FP32-rounded arrays, every level with a coarser one."""
    rng = np.random.default_rng(17)
    ctx = ctx_for(shape, precision=MG_MIXED)
    mg = O.MG(*shape, LAM, MU)
    for l in range(mg.levels - 1):
        d, dc = mg.dims(l), mg.dims(l + 1)
        x = rand_corner(rng, d).astype(np.float32).astype(np.float64)
        b = rand_corner(rng, d).astype(np.float32).astype(np.float64)
        if l > 0:
            x[:, [0, d[2]]] = 0
        bc = torch.zeros((3, dc[2] + 1, dc[1], dc[0]), dtype=torch.float32, device="cuda")
        ctx.residual_restrict32(l, g(b, torch.float32), g(x, torch.float32), bc)
        want = O.restrict(O.residual(mg.stencil(l), b, x))
        got = c(bc).astype(np.float64)
        assert np.isfinite(got).all()
        assert not got[:, [0, dc[2]]].any()  # wall planes untouched (zero)
        assert rel(got, want) <= 2e-6, (l, rel(got, want))
    ctx.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_residual_every_level(shape):
    rng = np.random.default_rng(1)
    ctx = ctx_for(shape)
    mg = O.MG(*shape, LAM, MU)
    for l in range(mg.levels):
        d = mg.dims(l)
        x = rand_corner(rng, d, walls=(l == 0))
        b = rand_corner(rng, d)
        r = torch.zeros_like(g(x))
        ctx.residual(l, g(b), g(x), r)
        want = O.residual(mg.stencil(l), b, x)
        assert rel(c(r), want) <= TOL64


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("descending", [False, True])
def test_smoother_fp64_every_level(shape, descending):
    rng = np.random.default_rng(2)
    ctx = ctx_for(shape)
    mg = O.MG(*shape, LAM, MU)
    for l in range(mg.levels):
        d = mg.dims(l)
        x = rand_corner(rng, d, walls=(l == 0))
        b = rand_corner(rng, d)
        xg = g(x)
        ctx.smooth(l, g(b), xg, 2, descending)
        S = mg.stencil(l)
        for _ in range(2):
            for col in (range(7, -1, -1) if descending else range(8)):
                O.gs_colour(S, b, x, col)
        assert rel(c(xg), x) <= TOL64


@pytest.mark.parametrize("shape", [(16, 16, 16), (24, 16, 8), (64, 64, 32)])
def test_smoother_fp32_fine_level(shape):
    rng = np.random.default_rng(3)
    ctx = ctx_for(shape, precision=MG_MIXED)
    mg = O.MG(*shape, LAM, MU)
    x = rand_corner(rng, shape, walls=False)
    b = rand_corner(rng, shape)
    x32 = x.astype(np.float32).astype(np.float64)
    b32 = b.astype(np.float32).astype(np.float64)
    xg = g(x32, torch.float32)
    ctx.smooth(0, g(b32, torch.float32), xg, 2, False)
    S = mg.stencil(0)
    for _ in range(2):
        for col in range(8):
            O.gs_colour(S, b32, x32, col)
    assert rel(c(xg), x32) <= 2e-6


# the bench's level shapes in miniature: finest rows of 128, 192 and 256
# nodes (persistent row strips), coarse rows of 128 (row strips with the
# 27-point operator), 64 x 64 coarse planes (27-point tile kernel), coarse
# planes of at most 32 x 32 nodes (whole-plane kernel)
FP32_LEVEL_SHAPES = [(256, 64, 32), (128, 128, 64), (192, 24, 16), (256, 32, 32)]


@pytest.mark.parametrize("shape", FP32_LEVEL_SHAPES)
@pytest.mark.parametrize("descending", [False, True])
@pytest.mark.parametrize("flags", [0, 1])
def test_smoother_fp32_every_level_against_oracle(shape, descending, flags):
    """Every FP32 sweep kernel the mixed solve runs at the bench's shapes
    (flags 0: the two-phase kernels; flags 1: eight colour launches) against
    the oracle's colour passes on the same FP32-rounded inputs, two sweeps,
    both colour orders, non-zero walls on the finest level."""
    rng = np.random.default_rng(31)
    ctx = ctx_for(shape, precision=MG_MIXED, flags=flags)
    mg = O.MG(*shape, LAM, MU)
    for l in range(mg.levels - 1):
        d = mg.dims(l)
        x = rand_corner(rng, d, walls=(l == 0)).astype(np.float32).astype(np.float64)
        b = rand_corner(rng, d).astype(np.float32).astype(np.float64)
        xg = g(x, torch.float32)
        ctx.smooth(l, g(b, torch.float32), xg, 2, descending)
        S = mg.stencil(l)
        for _ in range(2):
            for col in (range(7, -1, -1) if descending else range(8)):
                O.gs_colour(S, b, x, col)
        got = c(xg)
        assert np.array_equal(got[:, [0, d[2]]], x[:, [0, d[2]]])
        assert rel(got, x) <= 2e-6, (l, rel(got, x))
    ctx.close()


@pytest.mark.parametrize("shape", [(72, 40, 16), (16, 8, 12), (8, 4, 2), (136, 72, 32), (64, 32, 32),
                                   (10, 16, 16), (1024, 64, 64), (256, 32, 32), (128, 40, 32),
                                   (512, 32, 32), (192, 24, 16), (384, 32, 32), (768, 64, 64)])
@pytest.mark.parametrize("sweeps,descending", [(1, False), (2, False), (1, True), (3, True)])
def test_tiled_fp32_sweep_equals_colour_passes(shape, sweeps, descending):
    """The tiled two-phase FP32 sweeps reproduce the eight colour launches on
    every smoothed level (ragged tiles, odd sweep counts, non-zero walls on the
    finest level, both colour orders).  On the finest level rows of 64, 128,
    192 and 256 nodes take the persistent row-strip kernel, other rows of up
    to 512 nodes the per-tile row-strip kernel (136, 72, 384 and 512 wide),
    wider rows (768, 1024) the tile kernel; coarse levels take the row-strip
    kernel (rows of 128, 192 or 256 nodes, at least 9 rows), the whole-plane
    kernel (planes of at most 32 x 32 nodes) or the tile kernel."""
    rng = np.random.default_rng(7)
    ctxs = [ctx_for(shape, precision=MG_MIXED, flags=f) for f in (0, 1)]
    nlev = ctxs[0].levels
    for l in range(max(nlev - 1, 1)):
        nx, ny, nz = ctxs[0].level_dims(l)
        x = rng.uniform(-1, 1, (3, nz + 1, ny, nx)).astype(np.float32)
        if l > 0:
            x[:, 0] = 0
            x[:, nz] = 0
        b = rng.uniform(-1, 1, (3, nz + 1, ny, nx)).astype(np.float32)
        outs = []
        for ctx in ctxs:
            xg = g(x, torch.float32)
            ctx.smooth(l, g(b, torch.float32), xg, sweeps, descending)
            outs.append(c(xg))
        assert np.array_equal(outs[0][:, [0, nz]], x[:, [0, nz]])
        assert rel(outs[0], outs[1]) <= 1e-6, l
    for ctx in ctxs:
        ctx.close()


# finest grids whose rows the fused one-launch sweep takes: rows of 64-256
# nodes, ragged strips (ny = 40: 6 strips of 6 rows and one of 4), several
# CTAs per strip along z
FUSED_SHAPES = [(256, 32, 32), (128, 40, 32), (192, 24, 16), (64, 64, 64)]


@pytest.mark.parametrize("shape", FUSED_SHAPES)
@pytest.mark.parametrize("sweeps,descending", [(2, False), (3, True)])
def test_fused_sweep_equals_two_phase(shape, sweeps, descending):
    """The fused finest-level sweep (MG_FLAG_FUSED_SWEEP: both k-parities in
    one cooperative launch, ready flags between neighbouring strips) gives
    the two-launch sweep's result: every node update sees the same
    neighbour values, so the results agree to rounding (element-wise),
    non-zero walls included."""
    from paper_1904_03808_gb300.binding import MG_FLAG_FUSED_SWEEP
    rng = np.random.default_rng(13)
    nx, ny, nz = shape
    x = rng.uniform(-1, 1, (3, nz + 1, ny, nx)).astype(np.float32)
    b = rng.uniform(-1, 1, (3, nz + 1, ny, nx)).astype(np.float32)
    outs = []
    for flags in (MG_FLAG_FUSED_SWEEP, 0):
        ctx = ctx_for(shape, precision=MG_MIXED, flags=flags)
        xg = g(x, torch.float32)
        ctx.smooth(0, g(b, torch.float32), xg, sweeps, descending)
        outs.append(c(xg))
        ctx.close()
    assert np.array_equal(outs[0][:, [0, nz]], x[:, [0, nz]])
    assert rel(outs[0], outs[1]) <= 1e-6


@pytest.mark.parametrize("shape", SHAPES)
def test_restrict_and_prolong(shape):
    rng = np.random.default_rng(4)
    ctx = ctx_for(shape)
    mg = O.MG(*shape, LAM, MU)
    for l in range(mg.levels - 1):
        d, dc = mg.dims(l), mg.dims(l + 1)
        r = rand_corner(rng, d, walls=False)
        bc = torch.zeros((3, dc[2] + 1, dc[1], dc[0]), dtype=torch.float64, device="cuda")
        ctx.restrict(l, g(r), bc)
        assert rel(c(bc), O.restrict(r)) <= 1e-14
        xc = rand_corner(rng, dc, walls=False)
        x = rand_corner(rng, d)
        xg = g(x)
        ctx.prolong_add(l, g(xc), xg)
        O.prolong_add(xc, x)
        assert rel(c(xg), x) <= 1e-15


@pytest.mark.parametrize("shape", SHAPES)
def test_one_vcycle(shape):
    rng = np.random.default_rng(5)
    ctx = ctx_for(shape)
    mg = O.MG(*shape, LAM, MU)
    b = I.rhs_field(5, *shape)
    x = rand_corner(rng, shape)
    xg = g(x)
    ctx.vcycle(g(b), xg)
    mg.vcycle(b, x)
    assert rel(c(xg), x) <= TOL64


def _config1(n=32):
    b = I.rhs_field(1, n, n, n)
    v = np.zeros_like(b)
    v[0, 0], v[0, n] = -1.0, 1.0
    return b, v


@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 16, 8), (8, 12, 6), (64, 64, 64)])
def test_fp64_solve_matches_oracle_equal_cycles(shape):
    """Config: random RHS in [-1, 1), shear walls (-1, 0, 0)/(+1, 0, 0), v0 = 0;
    the oracle solves to 1e-10, the GPU runs the same number of V-cycles."""
    nx, ny, nz = shape
    b = I.rhs_field(1, nx, ny, nz)
    v = np.zeros_like(b)
    v[0, 0], v[0, nz] = -1.0, 1.0
    mg = O.MG(nx, ny, nz, LAM, MU)
    vo = v.copy()
    st, cyc, hist = mg.solve(b, vo, 1e-10, 100)
    assert st == 0
    ctx = ctx_for(shape, max_cycles=cyc)
    vg = g(v)
    st_g, s = ctx.solve(g(b), vg, tol=0.0)
    assert s.cycles == cyc
    assert rel(c(vg), vo) <= TOL64
    # residual histories: rounding of r = b - A v is ~eps |A| |v| per entry, so
    # late entries (near 1e-10) agree only to a few digits
    # (entries at the round-off floor, as after a direct solve on a single-level
    # grid, are compared in absolute terms)
    gh = np.array(s.resid_hist[:cyc + 1])
    big = hist > 1e-12
    assert np.allclose(gh[:4][big[:4]], hist[:4][big[:4]], rtol=1e-9, atol=0)
    assert np.allclose(gh[big], hist[big], rtol=5e-2, atol=0)
    assert np.all(gh[~big] <= 1e-12)
    # and to tolerance directly: the same cycle count up to a borderline cycle
    ctx2 = ctx_for(shape, max_cycles=100)
    vg2 = g(v)
    _, s2 = ctx2.solve(g(b), vg2, tol=1e-10)
    assert abs(s2.cycles - cyc) <= 1 and s2.rel_resid <= 1e-10


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 64, 64), (24, 16, 8)])
@pytest.mark.parametrize("inner", [0, 1, 3, 6])
def test_mixed_solve_reaches_tolerance(shape, inner):
    nx, ny, nz = shape
    b = I.rhs_field(1, nx, ny, nz)
    v = np.zeros_like(b)
    v[0, 0], v[0, nz] = -1.0, 1.0
    mg = O.MG(nx, ny, nz, LAM, MU)
    vo = v.copy()
    mg.solve(b, vo, 1e-12, 200)
    ctx = ctx_for(shape, precision=MG_MIXED, max_cycles=60, inner_cycles=inner)
    vg = g(v)
    st, s = ctx.solve(g(b), vg, tol=1e-10)
    assert st == 0 and s.rel_resid <= 1e-10
    # independent check of the reached residual with the oracle's operator
    vgn = c(vg)
    r = O.residual(mg.stencil(0), b, vgn)
    w = np.zeros_like(v)
    w[:, 0], w[:, nz] = v[:, 0], v[:, nz]
    bl = O.residual(mg.stencil(0), b, w)
    assert np.sqrt(O.norm2(r) / O.norm2(bl)) <= 1.05e-10
    err = rel(vgn, vo)
    assert err <= 1e-6, err


@pytest.mark.parametrize("shape", [(64, 64, 64), (256, 32, 32), (128, 48, 32)])
@pytest.mark.parametrize("flags", [0, 8])
def test_mixed_solve_fused_transfers(shape, flags):
    """The mixed solve with the finest level's residual and restriction fused
    into one row-strip pass (flags 0) and as separate passes (flags 8,
    MG_FLAG_UNFUSED_TRANSFERS): both reach the tolerance, checked
    with the oracle's operator, and stay within 1e-6 of the oracle's FP64
    solution (256 x 32 x 32 has a ragged last row strip)."""
    nx, ny, nz = shape
    b = I.rhs_field(2, nx, ny, nz)
    v = np.zeros_like(b)
    v[0, 0], v[0, nz] = -1.0, 1.0
    mg = O.MG(nx, ny, nz, LAM, MU)
    vo = v.copy()
    mg.solve(b, vo, 1e-12, 200)
    ctx = ctx_for(shape, precision=MG_MIXED, max_cycles=60, flags=flags)
    vg = g(v)
    st, s = ctx.solve(g(b), vg, tol=1e-10)
    assert st == 0 and s.rel_resid <= 1e-10
    vgn = c(vg)
    r = O.residual(mg.stencil(0), b, vgn)
    w = np.zeros_like(v)
    w[:, 0], w[:, nz] = v[:, 0], v[:, nz]
    bl = O.residual(mg.stencil(0), b, w)
    assert np.sqrt(O.norm2(r) / O.norm2(bl)) <= 1.05e-10
    assert rel(vgn, vo) <= 1e-6
    ctx.close()


@pytest.mark.parametrize("inner", [0, 4])
@pytest.mark.parametrize("shape,fused", [((32, 32, 32), 0), ((64, 64, 32), 4)])
def test_mixed_graph_replay_equals_direct_launches(inner, shape, fused):
    """The FP32 inner cycles replayed from CUDA graphs give bitwise the same
    iterate as the same kernels launched one by one (at 64 x 64 x 32 with
    the fused finest sweep: cooperative launches inside the graph)."""
    b = I.rhs_field(4, *shape)
    v = np.zeros_like(b)
    v[0, 0], v[0, shape[2]] = -1.0, 1.0
    outs = []
    for flags in (fused, 2 | fused):
        ctx = ctx_for(shape, precision=MG_MIXED, max_cycles=30, inner_cycles=inner, flags=flags)
        for _ in range(2):  # the second solve replays the captured graphs
            vg = g(v)
            st, s = ctx.solve(g(b), vg, tol=1e-10)
        outs.append((c(vg), s.cycles, s.outer_iters, s.rel_resid))
        ctx.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]


def test_zero_rhs_gives_zero_and_status_codes():
    shape = (16, 16, 16)
    ctx = ctx_for(shape, max_cycles=3)
    b = np.zeros((3, 17, 16, 16))
    x = np.ones_like(b)
    x[:, 0] = 0
    x[:, 16] = 0
    xg = g(x)
    st, s = ctx.solve(g(b), xg, tol=1e-10)
    assert st == 0 and s.cycles == 0 and float(xg.abs().max()) == 0.0
    # not converged within 3 cycles
    b = I.rhs_field(2, 16, 16, 16)
    st, s = ctx.solve(g(b), torch.zeros_like(g(b)), tol=1e-14, raise_on_error=False)
    assert st == 5 and s.cycles == 3
    # non-finite input
    b[1, 3, 2, 1] = np.nan
    st, s = ctx.solve(g(b), torch.zeros_like(g(b)), tol=1e-10, raise_on_error=False)
    assert st == 6
    # the context stays usable
    b = I.rhs_field(2, 16, 16, 16)
    st, s = ctx.solve(g(b), torch.zeros_like(g(b)), tol=0.0)
    assert st == 0 and s.cycles == 3


# --------------------------------------------------------------- step kernels

def _stz_state(n, nz=None, seed=3, preload=1.5e9):
    # strain 2% over 10 steps keeps chi physical (below ~700 K) in every test
    w = I.Workload(n, steps=10, strain=0.02, preload=preload, nz=nz, seed=seed)
    v, sig, chi, t = w.initial_state()
    rng = np.random.default_rng(seed)
    v[:, 1:w.nz] += 1e-3 * w.U_B * rng.normal(size=v[:, 1:w.nz].shape)
    sig += 5e7 * rng.normal(size=sig.shape)
    return w, v, sig, chi, t


@pytest.mark.parametrize("n,nz", [(16, None), (24, 8), (32, None)])
def test_pointwise_kernels(n, nz):
    w, v, sig, chi, t = _stz_state(n, nz)
    shape = (w.nx, w.ny, w.nz)
    ctx = ctx_for(shape, w=w)
    p = O.STZ(**w.stz)
    ss_o, D_o, sb_o = O.stress_star(v, sig, chi, w.h, w.dt, MU, p)
    assert (D_o > 0).mean() > 0.5  # plasticity active in most cells
    vg, sg, cg = g(v), g(sig), g(chi)
    ss, D, sb = torch.zeros_like(sg), torch.zeros_like(cg), torch.zeros_like(cg)
    ctx.stress_predict(vg, sg, cg, w.dt, ss, D, sb)
    assert rel(c(ss), ss_o) <= TOL64
    assert rel(c(D), D_o) <= TOL64 and rel(c(sb), sb_o) <= TOL64
    cn_o = O.chi_update(sig, chi, D_o, sb_o, w.h, w.dt, p)
    cn = torch.zeros_like(cg)
    ctx.chi_update(sg, cg, D, sb, w.dt, cn)
    assert rel(c(cn) - chi, cn_o - chi) <= 1e-10 and rel(c(cn), cn_o) <= TOL64
    b_o = O.div_rhs(ss_o, w.h, w.dt, MU)
    bg = torch.zeros_like(vg)
    ctx.rhs(ss, w.dt, bg)
    assert rel(c(bg), b_o) <= TOL64
    s_o = O.stress_final(v, ss_o, w.h, w.dt, LAM, MU)
    s1 = torch.zeros_like(sg)
    ctx.stress_correct(vg, ss, w.dt, s1)
    assert rel(c(s1), s_o) <= TOL64
    O.wall_fill(v, w.h, O.BC(**w.bc_values()), t + 3 * w.dt)
    ctx.wall_fill(vg, t + 3 * w.dt)
    assert np.array_equal(c(vg)[:, [0, w.nz]], v[:, [0, w.nz]])


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_disc_wall_fill(kind):
    n = 24
    w = I.Workload(n, steps=10, kind=kind)
    w.omega = 2 * np.pi / (1e8 * w.ts)
    ctx = ctx_for((n, n, n), w=w)
    v = np.zeros((3, n + 1, n, n))
    vg = g(v)
    ctx.wall_fill(vg, 5.0)
    O.wall_fill(v, w.h, O.BC(**w.bc_values()), 5.0)
    # exp() of the CUDA and C libraries may differ by an ulp, and a fused
    # multiply-add leaves ~1e-20 where x = -L + i h is exactly zero on the CPU
    assert np.allclose(c(vg), v, rtol=1e-13, atol=1e-13 * np.abs(v).max())


# multi-step runs use a 1.2 GPa preload: at 1.5 GPa the forward-Euler STZ
# update overshoots in the hottest cells (2 mu D dt / sbar > 2) and diverges
@pytest.mark.parametrize("preload,n,nz,steps", [(1.2e9, 16, None, 6), (0.0, 16, None, 4),
                                                 (1.2e9, 24, 8, 5), (1.2e9, 32, None, 4),
                                                 (1.2e9, 128, None, 2)])
def test_qs_step_trajectory(preload, n, nz, steps):
    """Whole steps, warm-started solves, FP64: the GPU runs the oracle's cycle
    count each step (tol = 0 with max_cycles = oracle cycles)."""
    w, v, sig, chi, t = _stz_state(n, nz, preload=preload)
    shape = (w.nx, w.ny, w.nz)
    mg = O.MG(*shape, LAM, MU)
    p = O.STZ(**w.stz)
    bc = O.BC(**w.bc_values())
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    for k in range(steps):
        st, cyc, hist = O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, p, bc, t, tol=1e-10,
                                  max_cycles=100)
        assert st == 0
        t += w.dt
        ctx = ctx_for(shape, w=w, max_cycles=cyc)
        st_g, s = ctx.step(state, w.dt, tol=0.0)
        assert s.cycles == cyc
        assert abs(state.t - t) <= 1e-15 * t and state.step == k + 1
        assert rel(c(vg), v) <= TOL64, k
        assert rel(c(sg), sig) <= TOL64, k
        assert rel(c(cg), chi) <= TOL64, k
        ctx.close()


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_qs_step_disc_walls_trajectory(kind):
    """Whole FP64 steps under the friction-welding walls of section 5 (kind 1:
    top disc rotating, bottom fixed; 2: both faces rotating together; 3:
    counter-rotating), chi0 with the section-5 recipe and a 1.2 GPa sigma_xz
    preload so that the STZ rate and the chi update are active, against the
    oracle with its cycle count each step."""
    import math
    n = 16
    w = I.Workload(n, steps=10, kind=kind, chi_mean=450.0, chi_std=15.0, lc_cells=2.0, seed=5,
                   dt_ts=2.0e3, preload=1.2e9)
    w.omega = 2.0 * math.pi / (1.0e8 * w.ts)
    v, sig, chi, t = w.initial_state()
    shape = (w.nx, w.ny, w.nz)
    mg = O.MG(*shape, LAM, MU)
    p = O.STZ(**w.stz)
    bc = O.BC(**w.bc_values())
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    for k in range(3):
        st, cyc, _ = O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, p, bc, t, tol=1e-10,
                               max_cycles=100)
        assert st == 0
        t += w.dt
        ctx = ctx_for(shape, w=w, max_cycles=cyc)
        ctx.step(state, w.dt, tol=0.0)
        ctx.close()
        assert rel(c(vg), v) <= TOL64, (kind, k)
        assert rel(c(sg), sig) <= TOL64, (kind, k)
        assert rel(c(cg), chi) <= TOL64, (kind, k)
    assert np.abs(v[:, w.nz]).max() > 0  # the top wall moved
    assert (np.abs(v[:, 0]).max() > 0) == (kind != 1)  # the bottom one with kinds 2, 3


@pytest.mark.parametrize("n,nz,steps", [(16, None, 4), (24, 8, 3), (32, None, 3)])
def test_qs_run_fused_steps(n, nz, steps):
    """qs_run: each step's stress correction and the next step's predictor run
    as one kernel.  FP64 with a fixed cycle count per step on both sides
    (tol = 0), against the oracle's steps and against separate qs_step calls."""
    w, v, sig, chi, t = _stz_state(n, nz, preload=1.2e9)
    shape = (w.nx, w.ny, w.nz)
    mg = O.MG(*shape, LAM, MU)
    p = O.STZ(**w.stz)
    bc = O.BC(**w.bc_values())
    cyc = 10
    v1, s1, c1 = g(v), g(sig), g(chi)
    v2, s2, c2 = g(v), g(sig), g(chi)
    run_state = make_state(v1, s1, c1, t)
    step_state = make_state(v2, s2, c2, t)
    for k in range(steps):
        st, n_o, _ = O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, p, bc, t, tol=0.0,
                               max_cycles=cyc)
        assert st == 0 and n_o == cyc
        t += w.dt
    ctx = ctx_for(shape, w=w, max_cycles=cyc)
    st, stats = ctx.run(run_state, steps, w.dt, tol=0.0)
    assert st == 0 and [s_.cycles for s_ in stats] == [cyc] * steps
    assert run_state.step == steps and abs(run_state.t - t) <= 1e-15 * t
    assert rel(c(v1), v) <= TOL64
    assert rel(c(s1), sig) <= TOL64
    assert rel(c(c1), chi) <= TOL64
    for _ in range(steps):
        ctx.step(step_state, w.dt, tol=0.0)
    # same arithmetic in the same order: equal up to contraction choices
    for a_, b_ in ((v1, v2), (s1, s2), (c1, c2)):
        assert rel(c(a_), c(b_)) <= 1e-14
    ctx.close()


def test_qs_run_edge_cases():
    """nsteps = 0 leaves the state alone; a solve that cannot converge stops
    the run after its (completed) step."""
    from paper_1904_03808_gb300 import binding
    w, v, sig, chi, t = _stz_state(16, preload=1.2e9)
    shape = (w.nx, w.ny, w.nz)
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    ctx = ctx_for(shape, w=w, max_cycles=1)
    st, stats = ctx.run(state, 0, w.dt)
    assert st == 0 and stats == [] and state.step == 0 and state.t == t
    assert np.array_equal(c(vg), v) and np.array_equal(c(sg), sig) and np.array_equal(c(cg), chi)
    st, stats = ctx.run(state, 3, w.dt, tol=1e-14, raise_on_error=False)
    assert st == binding.MG_ERR_NOCONV
    assert state.step == 1 and abs(state.t - (t + w.dt)) <= 1e-15 * t
    assert stats[0].cycles == 1 and stats[0].rel_resid > 1e-14
    # the stopped step is complete: its stress is the correction of its velocity
    assert np.isfinite(c(sg)).all() and not np.array_equal(c(sg), sig)
    assert ctx.run(state, -1, w.dt, raise_on_error=False)[0] == binding.MG_ERR_ARG
    ctx.close()


def test_qs_step_mixed_tracks_fp64():
    w, v, sig, chi, t = _stz_state(32, preload=1.2e9)
    shape = (w.nx, w.ny, w.nz)
    mg = O.MG(*shape, LAM, MU)
    p = O.STZ(**w.stz)
    bc = O.BC(**w.bc_values())
    ctx = ctx_for(shape, precision=MG_MIXED, w=w, max_cycles=40, inner_cycles=3)
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    for k in range(4):
        O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, p, bc, t, tol=1e-12, max_cycles=100)
        t += w.dt
        st, s = ctx.step(state, w.dt, tol=1e-10)
        assert st == 0 and s.rel_resid <= 1e-10
        ev, es = rel(c(vg), v), rel(c(sg), sig)
        assert ev <= 1e-6 and es <= 1e-6, (k, ev, es)


def test_fullsize_bench_step_256():
    """The bench's own configuration at full size: 256^3 cells, STZ-active
    preload, mixed precision, the bench's solver options, one warm-started
    step on the GPU.  The oracle then recomputes, from the same starting
    state, the intermediate stress, the right-hand side and the walls, and
    checks the GPU's velocity against its own operator (relative residual
    within the tolerance, lifted as in the stopping rule), its stress
    correction from that velocity and its chi update."""
    import bench
    w = bench.workload(256)
    v, sig, chi, t = w.initial_state()
    shape = (w.nx, w.ny, w.nz)
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    ctx = Context(*shape, w.h, I.TABLE1["K"], w.mu, bc=w.bc_values(), stz=w.stz,
                  precision=MG_MIXED, max_cycles=100, inner_cycles=bench.INNER)
    st, s = ctx.step(state, w.dt, bench.TOL)
    assert st == 0 and s.rel_resid <= bench.TOL
    ctx.close()
    p = O.STZ(**w.stz)
    bc = O.BC(**w.bc_values())
    ss, D, sb = O.stress_star(v, sig, chi, w.h, w.dt, MU, p)
    b = O.div_rhs(ss, w.h, w.dt, MU)
    vn = c(vg)
    vw = v.copy()
    O.wall_fill(vw, w.h, bc, t + w.dt)
    assert np.array_equal(vn[:, [0, w.nz]], vw[:, [0, w.nz]])
    S = O.fine_stencil(LAM, MU)
    v0 = vn.copy()
    v0[:, 1:w.nz] = 0.0
    bl2 = O.norm2(O.residual(S, b, v0))
    rel_resid = np.sqrt(O.norm2(O.residual(S, b, vn)) / bl2)
    # the library and the oracle sum the residual's 57 terms a node in
    # different orders: their values differ by at most a few ulps of
    # |A||v| + |b| a node, which bounds the difference of the two relative
    # residuals (the walls make |v| large against the lifted right-hand side)
    absS = np.abs(S)
    mag = O.apply(absS, np.abs(vn)) + np.abs(b)
    mag[:, [0, w.nz]] = 0.0
    floor = 64 * np.finfo(np.float64).eps * np.sqrt(O.norm2(mag) / bl2)
    assert abs(rel_resid - s.rel_resid) <= floor, (rel_resid, s.rel_resid, floor)
    assert rel_resid <= bench.TOL + floor, (rel_resid, floor)
    assert rel(c(sg), O.stress_final(vn, ss, w.h, w.dt, LAM, MU)) <= 1e-11
    assert rel(c(cg), O.chi_update(sig, chi, D, sb, w.h, w.dt, p)) <= 1e-12
