"""Pins of the oracle's pointwise step (sections 3.1, 3.3, 3.4, 4, 5):
staggered-difference exactness (Eq. 31), summation by parts between the
corner divergence and the cell gradient, the STZ rate against the Eq. (21)
form evaluated in high precision, the 0-D reduction of a whole step under
uniform simple shear, conservation and continuum consistency of the chi
diffusion term, the wall velocity profiles with their printed constants, and
the orthogonality of the projection in the energy inner product (section
2.4) to the order the collocated operator allows."""
import json
import math
import os

import mpmath as mp
import numpy as np
import pytest

import oracle as O
from paper_1904_03808_gb300 import inputs as I

MU = I.TABLE1["mu"]
LAM = I.lame_lambda(I.TABLE1["K"], MU)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def stz(l=1e-4):
    return O.STZ(**I.stz_values(l))


def test_cell_gradient_exact_on_trilinear():
    rng = np.random.default_rng(1)
    nx, ny, nz, h = 8, 6, 5, 0.3
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    X, Y, Z = i * h, j * h, k * h
    c = rng.normal(size=(3, 8))
    def f(a, X, Y, Z):
        return (c[a, 0] + c[a, 1] * X + c[a, 2] * Y + c[a, 3] * Z + c[a, 4] * X * Y +
                c[a, 5] * X * Z + c[a, 6] * Y * Z + c[a, 7] * X * Y * Z)
    v = np.stack([f(a, X, Y, Z) for a in range(3)])
    L = O.cell_gradient(v, h)
    kc, jc, ic = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    Xc, Yc, Zc = (ic + 0.5) * h, (jc + 0.5) * h, (kc + 0.5) * h
    sl = (slice(None), slice(0, ny - 1), slice(0, nx - 1))  # away from the periodic seam
    for a in range(3):
        dx = c[a, 1] + c[a, 4] * Yc + c[a, 5] * Zc + c[a, 7] * Yc * Zc
        dy = c[a, 2] + c[a, 4] * Xc + c[a, 6] * Zc + c[a, 7] * Xc * Zc
        dz = c[a, 3] + c[a, 5] * Xc + c[a, 6] * Yc + c[a, 7] * Xc * Yc
        for b, want in enumerate((dx, dy, dz)):
            assert np.allclose(L[..., a, b][sl], want[sl], rtol=1e-12, atol=1e-12)


def test_divergence_is_minus_gradient_transpose():
    """sum_corners v . div(sigma) = - sum_cells sigma : grad(v) for v with zero
    walls: the corner divergence and the Eq. (31) cell gradient are negative
    adjoints, which pins both index conventions."""
    rng = np.random.default_rng(2)
    nx, ny, nz, h, dt = 6, 8, 4, 0.7, 1.3
    v = rng.normal(size=(3, nz + 1, ny, nx))
    v[:, 0] = 0
    v[:, nz] = 0
    sig = rng.normal(size=(6, nz, ny, nx))
    b = O.div_rhs(sig, h, dt, MU) * (MU * dt / (h * h))  # undo the system scaling
    lhs = np.sum(v * b)
    L = O.cell_gradient(v, h)
    full = np.zeros((nz, ny, nx, 3, 3))
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3, (0, 2): 4, (2, 0): 4,
            (0, 1): 5, (1, 0): 5}
    for (a, bb), q in comp.items():
        full[..., a, bb] = sig[q]
    rhs = -np.sum(full * L)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


@pytest.mark.parametrize("sbar_gpa,chi", [(0.9, 600.0), (1.2, 600.0), (1.5, 600.0), (1.2, 690.0),
                                          (1.5, 900.0), (0.9, 900.0), (3.0, 450.0)])
def test_stz_rate_against_eq21_form(sbar_gpa, chi):
    """Eqs. (20)-(22): the oracle's cosh form equals C = (R(+s) + R(-s))/2 with
    R(+-s) = exp(-(Delta -+ Omega eps0 s)/(kB T)), evaluated here with 40 digits."""
    p = I.stz_values(1e-4)
    mp.mp.dps = 40
    s = mp.mpf(sbar_gpa) * mp.mpf(10) ** 9
    kT = mp.mpf(p["kB"]) * p["T"]
    dE = mp.mpf(p["Delta_K"]) * mp.mpf(p["kB"])
    b = mp.mpf(p["Omega"]) * p["eps0"] * s
    C = (mp.e ** (-(dE - b) / kT) + mp.e ** (-(dE + b) / kT)) / 2
    want = mp.e ** (-mp.mpf(p["ez_K"]) / chi) * C * (1 - mp.mpf(p["sY"]) / s) / p["tau0"]
    got = O.dpl(stz(), sbar_gpa * 1e9, chi)
    assert abs(got - float(want)) <= 1e-12 * float(want)


def test_stz_rate_yield_and_chi_scaling():
    p = stz()
    assert O.dpl(p, 0.85e9, 600.0) == 0.0
    assert O.dpl(p, 0.5e9, 900.0) == 0.0
    assert O.dpl(p, 1.2e9, 0.0) == 0.0
    r = O.dpl(p, 1.3e9, 650.0) / O.dpl(p, 1.3e9, 600.0)
    assert abs(r - math.exp(21000.0 * (1 / 600.0 - 1 / 650.0))) < 1e-12 * r


def _zero_d_reference(sig0, chi0, U_prev, U_next, H, dt, p):
    """One step of the per-cell ODE that the whole 3-D step reduces to when
    chi and sigma are uniform under simple shear: L = dv_x/dz = 2U/H in the
    (x, z) slot; Eq. (27) then Eq. (29) with D^{n+1} from U_next; Eq. (26)
    without diffusion (uniform fields)."""
    s = sig0
    Lm = np.zeros((3, 3))
    Lm[0, 2] = 2.0 * U_prev / H
    tr3 = np.trace(s) / 3.0
    s0 = s - tr3 * np.eye(3)
    sb = math.sqrt(0.5 * np.sum(s0 * s0))
    D = 0.0
    if sb > p["sY"]:
        kT = p["kB"] * p["T"]
        D = math.exp(-p["ez_K"] / chi0) * math.exp(-p["Delta_K"] / p["T"]) * \
            math.cosh(p["Omega"] * p["eps0"] * sb / kT) * (1 - p["sY"] / sb) / p["tau0"]
    plastic = (2 * MU * D / sb) * s0 if D > 0 else 0.0
    star = s + dt * (Lm @ s + s @ Lm.T - np.trace(Lm) * s - plastic)
    Dn = np.zeros((3, 3))
    Dn[0, 2] = Dn[2, 0] = U_next / H
    new = star + dt * (LAM * np.trace(Dn) * np.eye(3) + 2 * MU * Dn)
    chi1 = chi0 + dt / p["c0"] * (2 * D * sb / p["sY"]) * (p["chi_inf"] - chi0)
    return new, chi1


@pytest.mark.parametrize("preload", [0.0, 1.5e9])
def test_step_reduces_to_zero_d_under_uniform_shear(preload):
    n, steps = 8, 4
    w = I.Workload(n, steps=steps, strain=0.02, preload=preload)
    p = I.stz_values(w.h)
    v, sig, _, t = w.initial_state()
    chi = np.full((n, n, n), 640.0)
    mg = O.MG(n, n, n, LAM, MU)
    bc = O.BC(**w.bc_values())
    s_ref = np.zeros((3, 3))
    s_ref[0, 2] = s_ref[2, 0] = preload
    c_ref = 640.0
    def U(tt):
        return w.U_B * min(tt / w.t_ramp, 1.0)
    for _ in range(steps):
        st, cyc, hist = O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, O.STZ(**p), bc, t,
                                  tol=1e-13, max_cycles=200)
        assert st == 0
        s_ref, c_ref = _zero_d_reference(s_ref, c_ref, U(t), U(t + w.dt), w.H, w.dt, p)
        t += w.dt
        zk = (np.arange(n + 1) - n / 2.0) * w.h
        v_lin = 2.0 * U(t) / w.H * zk
        assert np.allclose(v[0], v_lin[:, None, None], rtol=0, atol=1e-10 * abs(U(t)))
        assert np.allclose(v[1:], 0.0, atol=1e-10 * abs(U(t)))
        comp = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
        scale = max(np.abs(s_ref).max(), 1.0)
        for q, (a, b) in enumerate(comp):
            assert np.allclose(sig[q], s_ref[a, b], rtol=0, atol=1e-9 * scale), (q, sig[q].ravel()[:2], s_ref[a, b])
        assert np.allclose(chi, c_ref, rtol=1e-13)
    if preload:
        assert c_ref > 640.0  # plasticity was active


def _x_wave_state(n, amp=20.0):
    h = 1e-4
    sig = np.zeros((6, 4, 4, n))
    sig[4] = 1.6e9
    x = (np.arange(n) + 0.5) / n
    chi = np.broadcast_to(650.0 + amp * np.sin(2 * np.pi * x), (4, 4, n)).copy()
    return h, sig, chi, x


def test_chi_diffusion_conserves_in_periodic_direction():
    p = stz(l=2e-4)
    n = 32
    h, sig, chi, _ = _x_wave_state(n)
    v = np.zeros((3, 5, 4, n))
    dt = 1e-6
    ss, D, sb = O.stress_star(v, sig, chi, h, dt, MU, p)
    new = O.chi_update(sig, chi, D, sb, h, dt, p)
    growth = dt / p.c0 * (2 * D * sb / p.sY) * (p.chi_inf - chi)
    diff = new - chi - growth
    row = diff[1, 1]
    # rounding of chi' - chi is ~eps * chi per cell; the telescoping sum is zero
    assert abs(row.sum()) <= 8 * np.finfo(float).eps * np.abs(chi).max() * n
    assert abs(row.sum()) <= 1e-8 * np.abs(row).sum()
    assert np.abs(row).max() > 0


def test_chi_diffusion_second_order_in_x():
    """l^2 d/dx(D dchi/dx) for chi = 650 + 20 sin(2 pi x/X), uniform stress:
    the discrete term converges at second order to the closed form
    l^2 (D' chi_x^2 + D chi_xx), D' = D e_z / chi^2."""
    p = stz()
    errs = []
    for n in (32, 64, 128):
        h, sig, chi, x = _x_wave_state(n)
        X = n * h
        p.l = 3e-5
        v = np.zeros((3, 5, 4, n))
        dt = 1e-6
        ss, D, sb = O.stress_star(v, sig, chi, h, dt, MU, p)
        new = O.chi_update(sig, chi, D, sb, h, dt, p)
        growth = dt / p.c0 * (2 * D * sb / p.sY) * (p.chi_inf - chi)
        term = (new - chi - growth)[1, 1] * p.c0 / dt
        c = chi[1, 1]
        cx = 20.0 * 2 * np.pi / X * np.cos(2 * np.pi * x)
        cxx = -20.0 * (2 * np.pi / X) ** 2 * np.sin(2 * np.pi * x)
        Dx = D[1, 1]
        want = p.l ** 2 * (Dx * p.ez_K / c ** 2 * cx ** 2 + Dx * cxx)
        errs.append(np.abs(term - want).max() / np.abs(want).max())
    assert abs(np.log2(errs[0] / errs[1]) - 2) < 0.15 and abs(np.log2(errs[1] / errs[2]) - 2) < 0.15, errs


def test_simple_shear_walls_and_ramp():
    n = 8
    v = np.zeros((3, n + 1, n, n))
    bc = O.BC(kind=0, U_B=2.0, t_ramp=4.0, omega=0, R=0, lambda_w=0)
    O.wall_fill(v, 0.1, bc, 1.0)
    assert np.all(v[0, n] == 0.5) and np.all(v[0, 0] == -0.5) and np.all(v[1:, [0, n]] == 0)
    O.wall_fill(v, 0.1, bc, 9.0)
    assert np.all(v[0, n] == 2.0) and np.all(v[0, 0] == -2.0)


def test_disc_walls_rotation():
    """Section 5: a rotation inside r < R with a smooth exp(-lambda_w (r^2-R^2)^2)
    cutoff; the printed choice of lambda_w leaves 10% of the angular velocity a
    quarter of the way from the disc edge to the domain edge."""
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    R = g["disc_R"]["value"]
    lam_w = 16 * math.log(10) / (1 - R * R) ** 2
    r2q = R * R + (1 - R * R) / 4
    assert abs(math.exp(-lam_w * (r2q - R * R) ** 2) - g["disc_quarter_way_fraction"]["value"]) < 1e-12
    n, h, om = 24, 1.0 / 12, 0.7
    v = np.zeros((3, n + 1, n, n))
    for kind, sgn in ((1, 0.0), (2, 1.0), (3, -1.0)):
        O.wall_fill(v, h, O.BC(kind=kind, U_B=0, t_ramp=1, omega=om, R=R, lambda_w=lam_w), 0.0)
        Lh = n * h / 2
        x = -Lh + np.arange(n) * h
        X, Y = np.meshgrid(x, x, indexing="xy")
        top = v[:, n]
        assert np.allclose(top[0] * X + top[1] * Y, 0.0, atol=1e-15)  # tangential
        r2 = (X ** 2 + Y ** 2) / Lh ** 2
        speed = np.hypot(top[0], top[1])
        inside = r2 < R * R
        assert np.allclose(speed[inside], om * np.sqrt(X ** 2 + Y ** 2)[inside], rtol=1e-14)
        f = speed[~inside] / (om * np.sqrt(X ** 2 + Y ** 2)[~inside])
        assert np.all(f <= 1) and np.all(f >= 0) and f.min() < 1e-30
        assert np.all(top[2] == 0)
        assert np.allclose(v[:, 0], sgn * top, atol=0)


def test_printed_constants():
    """Table 1 and section 4: c_s = sqrt(mu/rho) = 2.47 km/s, t_s = L/c_s = 4.05 us."""
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    cs = math.sqrt(g["mu"]["value"] / g["rho"]["value"])
    assert round(cs / 1000, 2) == g["c_s_km_per_s"]["value"]
    ts = g["L"]["value"] / cs
    assert round(ts * 1e6, 2) == g["t_s_us"]["value"]
    assert abs(I.shear_time_unit() - ts) < 1e-18
    for key in ("K", "mu", "rho", "sY", "tau0", "eps0", "c0", "Delta_K", "T", "chi_inf", "ez_K"):
        assert I.TABLE1[key] == g[key]["value"], key
    assert abs(I.TABLE1["Omega"] - g["Omega_A3"]["value"] * 1e-30) < 1e-40


def test_chi_diffusion_second_order_at_the_z_walls():
    """Fields linear in z -- chi = 620 + 30 z/Z and sigma_xz = 1.5 + 0.2 z/Z GPa,
    uniform in x and y, above yield -- continue exactly by linear
    extrapolation, so the ghost cells beyond the walls (extrapolated chi and
    sigma, D^pl taken from the extrapolated values: reading of section 4) give
    the first and last cells the stencil of an interior cell.  The discrete
    l^2 d/dz(D dchi/dz) must then converge at second order to the closed form
    l^2 chi_z dD/dz in every cell, the wall cells included; a wrong ghost
    value or index, or a ghost D^pl taken from the unextrapolated fields,
    leaves an O(1) or O(h) error there.  dD/dz is a fine 5-point difference of
    the pointwise rate D(sbar(z), chi(z)) along the exact fields."""
    p = stz(l=1e-4)
    dt = 1e-5
    errs, errs_wall = [], []
    for n in (16, 32, 64):
        h = 1e-4
        Z = n * h
        z = (np.arange(n) + 0.5) * h
        chi_f = lambda zz: 620.0 + 30.0 * zz / Z  # noqa: E731
        sig_f = lambda zz: 1.5e9 + 0.2e9 * zz / Z  # noqa: E731
        chi = np.broadcast_to(chi_f(z)[:, None, None], (n, 4, 4)).copy()
        sig = np.zeros((6, n, 4, 4))
        sig[4] = sig_f(z)[:, None, None]
        v = np.zeros((3, n + 1, 4, 4))
        ss, D, sb = O.stress_star(v, sig, chi, h, dt, MU, p)
        new = O.chi_update(sig, chi, D, sb, h, dt, p)
        growth = dt / p.c0 * (2 * D * sb / p.sY) * (p.chi_inf - chi)
        term = ((new - chi - growth) * p.c0 / dt)[:, 1, 1]
        # sbar of a pure xz shear is |sigma_xz|
        rate = lambda zz: O.dpl(p, sig_f(zz), chi_f(zz))  # noqa: E731
        dlt = Z * 1e-4
        want = np.array([p.l ** 2 * (30.0 / Z) *
                         (-rate(zz + 2 * dlt) + 8 * rate(zz + dlt) - 8 * rate(zz - dlt) +
                          rate(zz - 2 * dlt)) / (12 * dlt) for zz in z])
        assert np.allclose(D[:, 1, 1], [rate(zz) for zz in z], rtol=1e-12, atol=0)
        err = np.abs(term - want) / np.abs(want).max()
        errs.append(err.max())
        errs_wall.append(max(err[0], err[-1]))
    for e in (errs, errs_wall):
        assert abs(np.log2(e[0] / e[1]) - 2) < 0.2 and abs(np.log2(e[1] / e[2]) - 2) < 0.2, e


def _linear_velocity(L, nx, ny, nz, h):
    """Corner velocities v_a = sum_b L_ab x_b (x_b = index * h)."""
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    X = [i * h, j * h, k * h]
    return np.stack([sum(L[a, b] * X[b] for b in range(3)) for a in range(3)])


def test_stress_predictor_under_linear_velocity():
    """Below yield (D^pl = 0) and for a velocity linear in x, y, z, every
    cell away from the periodic wrap sees the constant gradient L, and Eq. 27
    gives sigma* = sigma + dt (L sigma + sigma L^T - tr(L) sigma) for a
    general L and a general symmetric sigma (all six components)."""
    rng = np.random.default_rng(12)
    nx, ny, nz, h, dt = 7, 6, 5, 1e-3, 1e-2
    L = rng.normal(size=(3, 3))
    v = _linear_velocity(L, nx, ny, nz, h)
    S = rng.normal(size=(3, 3)) * 1e8
    S = 0.5 * (S + S.T)  # ~0.1 GPa: far below the 0.85 GPa yield stress
    comp = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    sig = np.stack([np.full((nz, ny, nx), S[a, b]) for a, b in comp])
    chi = np.full((nz, ny, nx), 600.0)
    ss, D, _ = O.stress_star(v, sig, chi, h, dt, MU, stz())
    assert np.all(D == 0.0)
    want = S + dt * (L @ S + S @ L.T - np.trace(L) * S)
    for q, (a, b) in enumerate(comp):
        got = ss[q][:, : ny - 1, : nx - 1]  # cells whose corners do not wrap
        assert np.allclose(got, want[a, b], rtol=0, atol=1e-12 * np.abs(S).max()), (a, b)


def test_stress_predictor_rotation_keeps_invariants():
    """A rigid rotation rate (L = W skew, tr W = 0) leaves tr(sigma*) =
    tr(sigma) to rounding and changes |sigma|_F^2 only at second order in dt
    (the rate W sigma - sigma W is orthogonal to sigma)."""
    rng = np.random.default_rng(13)
    nx, ny, nz, h = 6, 6, 4, 1e-3
    w = rng.normal(size=3)
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    v = _linear_velocity(W, nx, ny, nz, h)
    S = rng.normal(size=(3, 3)) * 1e8
    S = 0.5 * (S + S.T)
    comp = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    sig = np.stack([np.full((nz, ny, nx), S[a, b]) for a, b in comp])
    chi = np.full((nz, ny, nx), 600.0)
    for dt in (1e-2, 5e-3):
        ss, _, _ = O.stress_star(v, sig, chi, h, dt, MU, stz())
        c = (slice(None), slice(0, ny - 1), slice(0, nx - 1))
        tr0, tr1 = np.trace(S), ss[0][c] + ss[1][c] + ss[2][c]
        assert np.allclose(tr1, tr0, rtol=0, atol=1e-13 * np.abs(S).max())
        f2 = ss[0][c] ** 2 + ss[1][c] ** 2 + ss[2][c] ** 2 + 2 * (
            ss[3][c] ** 2 + ss[4][c] ** 2 + ss[5][c] ** 2)
        R = W @ S - S @ W
        assert np.allclose(f2 - np.sum(S * S), dt ** 2 * np.sum(R * R), rtol=1e-6, atol=0)


def _compliance(t):
    # S = C^-1 for the isotropic C (lambda, mu) on stored components
    # xx, yy, zz, yz, xz, xy
    out = t / (2.0 * MU)
    tr = (t[0] + t[1] + t[2]) * LAM / (2.0 * MU * (3.0 * LAM + 2.0 * MU))
    for a in range(3):
        out[a] = out[a] - tr
    return out


def _energy_inner(a, b, h):
    # <a, b> = sum over cells of a : S : b h^3 (Eq. 18)
    Sb = _compliance(b)
    w = (1.0, 1.0, 1.0, 2.0, 2.0, 2.0)
    return h ** 3 * sum(w[q] * float(np.sum(a[q] * Sb[q])) for q in range(6))


def _projection_cosine(n, flip=False):
    # sigma^n = 0 and fixed walls: project a smooth sigma* (Eqs. 28-30) and
    # return |<sigma^{n+1} - sigma^n, sigma^{n+1} - sigma*>| over the product
    # of the two norms
    L = 0.01
    h = 2.0 * L / n
    dt = 200.0 * I.shear_time_unit(L)
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    px, py, pz = 2 * np.pi * X, 2 * np.pi * Y, np.pi * Z
    ss = 1e8 * np.stack([np.sin(px + 0.3) * np.cos(py) * np.cos(pz),
                         np.cos(px) * np.sin(2 * py + 0.1) * np.sin(pz),
                         np.sin(px - py) * np.cos(2 * pz),
                         np.cos(2 * px) * np.cos(py + 0.5) * np.sin(pz + 0.2),
                         np.sin(px + 2 * py) * np.cos(pz),
                         np.cos(px - 0.4) * np.sin(py) * np.sin(2 * pz)])
    mg = O.MG(n, n, n, LAM, MU)
    v = np.zeros((3, n + 1, n, n))
    st, _, _ = mg.solve(O.div_rhs(ss, h, dt, MU), v, tol=1e-13, max_cycles=200)
    assert st == 0
    s1 = O.stress_final(v, ss, h, dt, LAM, MU)
    d = s1 - ss
    if flip:  # a planted sign error in the stress correction
        s1, d = ss - d, -d
    return abs(_energy_inner(s1, d, h)) / math.sqrt(_energy_inner(s1, s1, h) *
                                                     _energy_inner(d, d, h))


def test_projection_is_orthogonal_in_the_energy_inner_product():
    """Section 2.4, Eqs. 18-19: the projection is orthogonal in the
    compliance-weighted inner product, <sigma^{n+1} - sigma^n, sigma^{n+1} -
    sigma*> = 0.  The operator solved here is the collocated one (Eqs. 32
    and 34), not the composition
    of the staggered divergence and gradient, so the discrete projection is
    orthogonal only to O(h^2): the cosine of the angle falls by about 4 per
    halving of h.  A sign error in the correction leaves it of order one."""
    eye = np.zeros((6, 1, 1, 1))
    eye[:3] = 1.0
    t = np.random.default_rng(3).normal(size=(6, 1, 1, 1))
    C_t = 2.0 * MU * t + LAM * (t[0] + t[1] + t[2]) * eye
    assert np.allclose(_compliance(C_t), t, rtol=1e-14, atol=1e-14 * np.abs(t).max())
    r = [_projection_cosine(n) for n in (16, 32, 64)]
    assert r[2] < 0.01
    assert 0.2 < r[1] / r[0] < 0.33 and 0.2 < r[2] / r[1] < 0.3, r
    assert _projection_cosine(16, flip=True) > 0.5
