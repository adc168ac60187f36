"""Pins of the oracle's projection operator (Eq. 30 with the stencils of
section 3.4) and its multigrid transfers (section 3.6), each against something
other than the oracle itself: exactness on polynomials, the closed-form
Fourier symbol, an independent Kronecker-product assembly, symmetry / SPD
(the paper's condition B) and the loss of diagonal dominance (condition A).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1904_03808_gb300 import inputs as I

K, MU = I.TABLE1["K"], I.TABLE1["mu"]
LAM = I.lame_lambda(K, MU)
KAP = (LAM + MU) / MU
LP = (LAM + 2 * MU) / MU


def test_scaled_diagonal_value():
    # diagonal of -(h^2/(mu dt)) A is (2 lam + 8 mu)/mu
    S = O.fine_stencil(LAM, MU)
    assert np.allclose(np.diag(S[13]), (2 * LAM + 8 * MU) / MU, rtol=0, atol=1e-14)
    assert abs(S[13, 0, 0] - 13.190730837789661) < 1e-12


def _grid(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    return i.astype(float), j.astype(float), k.astype(float)


def test_exact_on_quadratics():
    """The collocated 3-point and 4-point stencils are exact on quadratics:
    A v equals -(1/mu)[(lam+2mu) v_a,aa + mu sum v_a,bb + (lam+mu) sum v_b,ab]."""
    rng = np.random.default_rng(0)
    nx, ny, nz = 8, 8, 6
    x, y, z = _grid(nx, ny, nz)
    X = [x, y, z]
    v = np.zeros((3, nz + 1, ny, nx))
    H = np.zeros((3, 3, 3))  # Hessian of each component
    for a in range(3):
        Q = rng.normal(size=(3, 3))
        Q = Q + Q.T
        lin = rng.normal(size=3)
        v[a] = 0.5 * sum(Q[p, q] * X[p] * X[q] for p in range(3) for q in range(3)) + \
            sum(lin[p] * X[p] for p in range(3)) + rng.normal()
        H[a] = Q
    Av = O.apply(O.fine_stencil(LAM, MU), v)
    for a in range(3):
        want = (LAM + 2 * MU) * H[a, a, a] + MU * sum(H[a, b, b] for b in range(3) if b != a) + \
            (LAM + MU) * sum(H[b, a, b] for b in range(3) if b != a)
        want = -want / MU
        got = Av[a, 1:nz, 1:ny - 1, 1:nx - 1]  # away from the periodic seam
        assert np.allclose(got, want, rtol=1e-10, atol=1e-8 * np.abs(v).max())


def _symbol(theta):
    s = np.sin(np.asarray(theta) / 2)
    c = np.cos(np.asarray(theta) / 2)
    Kc = np.outer(c, c)
    np.fill_diagonal(Kc, 1.0)
    S = np.diag(s)
    return 4 * np.sum(s * s) * np.eye(3) + KAP * 4 * S @ Kc @ S


@pytest.mark.parametrize("seed", range(4))
def test_fourier_symbol(seed):
    """Single Fourier modes are eigenvectors of the operator; the symbol is
    4 sum s_j^2 I + ((lam+mu)/mu) 4 S K S, s_j = sin(theta_j/2)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = 8, 12, 6
    m = (rng.integers(0, nx), rng.integers(0, ny))
    theta = np.array([2 * np.pi * m[0] / nx, 2 * np.pi * m[1] / ny, rng.uniform(0, np.pi)])
    chat = rng.normal(size=3) + 1j * rng.normal(size=3)
    x, y, z = _grid(nx, ny, nz)
    ph = np.exp(1j * (theta[0] * x + theta[1] * y + theta[2] * z))
    v = np.stack([np.real(chat[a] * ph) for a in range(3)])
    Av = O.apply(O.fine_stencil(LAM, MU), v)
    Mc = _symbol(theta) @ chat
    for a in range(3):
        want = np.real(Mc[a] * ph)[1:nz]
        assert np.allclose(Av[a, 1:nz], want, rtol=0, atol=1e-12 * np.abs(chat).max() * 20)


def test_symbol_fails_for_planted_sign_error():
    """A plausible mistake (mixed-term sign flipped) is caught by the symbol."""
    S = O.fine_stencil(LAM, MU).copy()
    for d in range(27):
        if d != 13:
            off = S[d] - np.diag(np.diag(S[d]))
            S[d] = np.diag(np.diag(S[d])) - off
    nx, ny, nz = 8, 8, 6
    x, y, z = _grid(nx, ny, nz)
    theta = np.array([2 * np.pi / 8, 2 * np.pi * 3 / 8, 0.9])
    chat = np.array([1.0, 2.0, -1.0])
    ph = np.exp(1j * (theta[0] * x + theta[1] * y + theta[2] * z))
    v = np.stack([np.real(chat[a] * ph) for a in range(3)])
    Av = O.apply(S, v)
    want = np.real((_symbol(theta) @ chat)[0] * ph)[1:nz]
    assert not np.allclose(Av[0, 1:nz], want, atol=1e-6)


# --- independent Kronecker assembly -------------------------------------

def _d2_periodic(n):
    return sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1], format="lil") + \
        sp.coo_matrix(([1.0, 1.0], ([0, n - 1], [n - 1, 0])), shape=(n, n))


def _d1_periodic(n):
    m = sp.lil_matrix((n, n))
    for i in range(n):
        m[i, (i + 1) % n] += 0.5
        m[i, (i - 1) % n] -= 0.5
    return m.tocsr()


def _dz_full(nz, order):
    """(nz-1) x (nz+1): interior rows, all planes as columns."""
    m = sp.lil_matrix((nz - 1, nz + 1))
    for r, k in enumerate(range(1, nz)):
        if order == 2:
            m[r, k - 1] += 1
            m[r, k] -= 2
            m[r, k + 1] += 1
        else:
            m[r, k + 1] += 0.5
            m[r, k - 1] -= 0.5
    return m.tocsr()


def kron_operator(nx, ny, nz):
    """Scaled operator Ahat = -(1/mu)[...] on interior rows x all-plane
    columns, component-major, built from 1-D stencils by Kronecker products."""
    Ix, Iy = sp.identity(nx), sp.identity(ny)
    Izf = sp.eye(nz - 1, nz + 1, k=1)  # interior rows pick their own plane
    D2 = [sp.kron(Izf, sp.kron(Iy, _d2_periodic(nx))),
          sp.kron(Izf, sp.kron(_d2_periodic(ny), Ix)),
          sp.kron(_dz_full(nz, 2), sp.kron(Iy, Ix))]
    D1 = [(Izf, Iy, _d1_periodic(nx)), (Izf, _d1_periodic(ny), Ix), (_dz_full(nz, 1), Iy, Ix)]

    def mixed(a, b):
        f = [D1[0][0] if 2 not in (a, b) else D1[2][0],
             _d1_periodic(ny) if 1 in (a, b) else Iy,
             _d1_periodic(nx) if 0 in (a, b) else Ix]
        return sp.kron(f[0], sp.kron(f[1], f[2]))

    blocks = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            if a == b:
                blk = (LAM + 2 * MU) * D2[a] + MU * sum(D2[c] for c in range(3) if c != a)
            else:
                blk = (LAM + MU) * mixed(a, b)
            blocks[a][b] = -blk / MU
    return sp.bmat(blocks).tocsr()


def _interior_cols(nx, ny, nz):
    n_all = (nz + 1) * ny * nx
    idx = np.arange(3 * n_all).reshape(3, nz + 1, ny, nx)
    return idx[:, 1:nz].ravel()


def test_apply_matches_kronecker_assembly():
    rng = np.random.default_rng(3)
    nx, ny, nz = 6, 8, 6
    A = kron_operator(nx, ny, nz)
    v = rng.normal(size=(3, nz + 1, ny, nx))
    Av = O.apply(O.fine_stencil(LAM, MU), v)
    want = (A @ v.ravel()).reshape(3, nz - 1, ny, nx)
    assert np.allclose(Av[:, 1:nz], want, rtol=1e-14, atol=1e-13)
    assert np.all(Av[:, 0] == 0) and np.all(Av[:, nz] == 0)


def _nm_perm(nx, ny, nz):
    """component-major interior index -> oracle's node-major index"""
    nn = (nz - 1) * ny * nx
    cm = np.arange(3 * nn)
    a, node = cm // nn, cm % nn
    return node * 3 + a


def test_dense_matches_kronecker_and_is_spd():
    nx = ny = nz = 8
    mg = O.MG(nx, ny, nz, LAM, MU)
    D = mg.dense(0)
    p = _nm_perm(nx, ny, nz)
    Akr = kron_operator(nx, ny, nz)[:, _interior_cols(nx, ny, nz)].toarray()
    assert np.allclose(D[np.ix_(p, p)], Akr, rtol=0, atol=1e-13)
    assert np.array_equal(D, D.T)  # fine stencil is exactly symmetric
    w = np.linalg.eigvalsh(D)
    assert w.min() > 0  # condition B of section 3.3: SPD
    np.linalg.cholesky(D)
    # condition A of section 3.3 fails: rows away from the walls are not
    # diagonally dominant (off-diagonal sum (4 lam + 10 mu)/mu > (2 lam + 8 mu)/mu)
    off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    fails = off > np.abs(np.diag(D)) + 1e-12
    assert fails.sum() >= 3 * nx * ny * (nz - 3)
    assert np.isclose(off.max(), (4 * LAM + 10 * MU) / MU)


def _t_periodic(nf):
    m = sp.lil_matrix((nf, nf // 2))
    for I_ in range(nf // 2):
        m[2 * I_, I_] = 1.0
        m[(2 * I_ + 1) % nf, I_] += 0.5
        m[(2 * I_ - 1) % nf, I_] += 0.5
    return m.tocsr()


def _t_wall(nzf):
    """fine interior planes 1..nzf-1 x coarse interior planes 1..nzf/2-1"""
    m = sp.lil_matrix((nzf - 1, nzf // 2 - 1))
    for c, K_ in enumerate(range(1, nzf // 2)):
        m[2 * K_ - 1, c] = 1.0
        m[2 * K_ - 2, c] = 0.5
        m[2 * K_, c] = 0.5
    return m.tocsr()


def kron_T(nx, ny, nz):
    t = sp.kron(_t_wall(nz), sp.kron(_t_periodic(ny), _t_periodic(nx)))
    return sp.kron(sp.identity(3), t).tocsr()  # component-major


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 8, 8), (8, 12, 16)])
def test_galerkin_equals_explicit_triple_product(shape):
    """Eq. (36): the coarse operator equals R A T with R = T^T, built here from
    1-D linear interpolation matrices, and is one constant 27-point stencil."""
    nx, ny, nz = shape
    mg = O.MG(nx, ny, nz, LAM, MU)
    T = kron_T(nx, ny, nz)
    Af = mg.dense(0)
    p = _nm_perm(nx, ny, nz)
    Af_cm = Af[np.ix_(p, p)]
    Ac = (T.T @ (T.T @ Af_cm.T).T)  # T^T A T
    Ac = np.asarray(Ac)
    cx, cy, cz = nx // 2, ny // 2, nz // 2
    pc = _nm_perm(cx, cy, cz)
    Dc = mg.dense(1)[np.ix_(pc, pc)]
    assert np.allclose(Dc, Ac, rtol=0, atol=1e-13 * np.abs(Ac).max())
    assert np.allclose(Dc, Dc.T, rtol=0, atol=1e-14 * np.abs(Dc).max())
    assert np.linalg.eigvalsh(Dc).min() > 0


def test_restrict_and_prolong_are_T_transpose_and_T():
    rng = np.random.default_rng(5)
    nx, ny, nz = 8, 12, 8
    T = kron_T(nx, ny, nz)
    r = rng.normal(size=(3, nz + 1, ny, nx))
    r[:, 0] = 0
    r[:, nz] = 0
    bc = O.restrict(r)
    want = T.T @ r[:, 1:nz].ravel()
    assert np.allclose(bc[:, 1:nz // 2].ravel(), want, rtol=1e-14, atol=1e-14)
    assert np.all(bc[:, 0] == 0) and np.all(bc[:, nz // 2] == 0)
    xc = rng.normal(size=(3, nz // 2 + 1, ny // 2, nx // 2))
    xc[:, 0] = 0
    xc[:, nz // 2] = 0
    x = rng.normal(size=(3, nz + 1, ny, nx))
    x0 = x.copy()
    O.prolong_add(xc, x)
    want = T @ xc[:, 1:nz // 2].ravel()
    assert np.allclose((x - x0)[:, 1:nz].ravel(), want, rtol=1e-14, atol=1e-14)
    assert np.array_equal(x[:, 0], x0[:, 0]) and np.array_equal(x[:, nz], x0[:, nz])


def test_same_colour_nodes_do_not_couple():
    """8-colour ordering: every nonzero offset of the 27-point stencil changes
    the parity of at least one index, so a colour pass is order-independent;
    checked by brute-force block Gauss-Seidel on the dense matrix."""
    rng = np.random.default_rng(7)
    nx, ny, nz = 4, 4, 6
    mg = O.MG(nx, ny, nz, LAM, MU)
    for lvl_S in (mg.stencil(0), O.galerkin(mg.stencil(0))):
        b = rng.normal(size=(3, nz + 1, ny, nx))
        x = rng.normal(size=(3, nz + 1, ny, nx))
        xo = x.copy()
        for c in range(8):
            O.gs_colour(lvl_S, b, xo, c)
        # brute force: node-by-node block solves straight from the stencil
        xb = x.copy()
        for c in range(8):
            nodes = [(k, j, i) for k in range(1, nz) for j in range(ny) for i in range(nx)
                     if (i & 1) + 2 * (j & 1) + 4 * (k & 1) == c]
            for (k, j, i) in reversed(nodes):  # any order inside a colour
                f = b[:, k, j, i].copy()
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
                            if d == 13:
                                continue
                            f -= lvl_S[d] @ xb[:, k + dz, (j + dy) % ny, (i + dx) % nx]
                xb[:, k, j, i] = np.linalg.solve(lvl_S[13], f)
        assert np.allclose(xo, xb, rtol=1e-13, atol=1e-13)


def test_galerkin_stencils_keep_the_reflection_symmetry():
    """Reflecting one axis maps the elastic problem of Eq. (30) onto itself
    with that velocity component negated, and trilinear T commutes with the
    reflection, so every Galerkin level (Eq. 36) keeps the fine stencil's
    parity structure: with A(d) the 3x3 block of offset d = (dx, dy, dz),
      - A(d)_aa is even in each of dx, dy, dz;
      - A(d)_ab (a != b) is odd in d_a and in d_b and even in the third
        offset, hence zero unless d_a and d_b are both non-zero (153 of the
        243 entries can be non-zero);
      - A(-d) = A(d)^T.
    Checked on the fine stencil and six Galerkin levels (the coarse kernels
    store one coefficient per parity class: 21 diagonal and 6 coupling)."""
    S = O.fine_stencil(LAM, MU)
    for level in range(7):
        T = S.reshape(3, 3, 3, 3, 3)  # [dz+1, dy+1, dx+1, a, b]
        scale = np.abs(S).max()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    d = (dx, dy, dz)
                    A = T[dz + 1, dy + 1, dx + 1]
                    assert np.allclose(A, T[1 - dz, 1 - dy, 1 - dx].T, rtol=0, atol=1e-14 * scale)
                    for a in range(3):
                        for b in range(3):
                            # flip each axis in turn
                            for ax in range(3):
                                e = list(d)
                                e[ax] = -e[ax]
                                Ae = T[e[2] + 1, e[1] + 1, e[0] + 1]
                                sign = (-1 if ax == a else 1) * (-1 if ax == b else 1)
                                assert abs(Ae[a, b] - sign * A[a, b]) <= 1e-14 * scale, \
                                    (level, d, a, b, ax)
                            if a != b and (d[a] == 0 or d[b] == 0):
                                assert abs(A[a, b]) <= 1e-14 * scale, (level, d, a, b)
        nz = sum(1 for v in S.ravel() if abs(v) > 1e-14 * np.abs(S).max())
        assert nz <= 153
        if level >= 1:
            assert nz == 153  # every admissible coupling appears on coarse levels
        S = O.galerkin(S)
