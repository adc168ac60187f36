"""Gradient oracle: the derivative of the plastic work of a run of
quasi-static projection steps with respect to the initial effective
temperature chi^0.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only tests import it.

The objective is not one the paper evaluates; it is the total plastic work
of K steps,

    W = sum_n sum_cells 2 D^pl_n sbar_n dt h^3,

(D^pl : sigma_0 = 2 D^pl sbar is the plastic power per unit volume, the
growth term of Eq. 26), and its gradient dW/dchi^0 is the plain definition:
the chain rule through every step.  This module restates the step of
section 3.3 in plain PyTorch FP64 CPU operations, one function per equation
of the C oracle, so that autograd differentiates exactly what is written:

  - cell gradient, Eq. (31), x and y periodic;
  - sbar from the deviatoric stress (section 3.1) and the athermal STZ rate,
    Eqs. (20)-(22), zero at or below yield (its subgradient there is 0);
  - intermediate stress, Eq. (27);
  - effective temperature, Eq. (26), conservative 7-point diffusion with
    face-averaged D^pl and linearly extrapolated z ghost cells;
  - right-hand side (h^2/(mu dt)) div sigma*, the corner version of Eq. (31);
  - the projection solve of Eq. (30) by the C oracle's multigrid, wrapped so
    that its derivative is the solve of the same symmetric operator (the
    scaled operator is symmetric, so the adjoint of v = A^-1 b is
    b_bar = A^-1 v_bar, with zero walls: the wall values do not depend on
    chi^0);
  - stress correction, Eq. (29).

``step`` agrees with the C oracle's ``qs_step`` to rounding (a test pins
this), and the gradient is pinned by central finite differences of the
C oracle's own forward run.
"""
from __future__ import annotations

import math

import torch

from . import MG, wall_fill

_F64 = torch.float64
# stress component index of sigma_ab in the stored order xx, yy, zz, yz, xz, xy
_COMP = ((0, 5, 4), (5, 1, 3), (4, 3, 2))


def _full(s6):
    """(6, ...) stored components -> (3, 3, ...) symmetric tensor."""
    return torch.stack([torch.stack([s6[_COMP[a][b]] for b in range(3)]) for a in range(3)])


def _stored(s):
    """(3, 3, ...) -> (6, ...) in the stored order."""
    return torch.stack([s[0, 0], s[1, 1], s[2, 2], s[1, 2], s[0, 2], s[0, 1]])


def cell_gradient(v, h):
    """Eq. (31): L[a, b] = d v_a / d x_b at the cell centres, (3, 3, nz, ny, nx),
    from the 8 corners of each cell; x and y wrap."""
    rows = []
    for a in range(3):
        V = v[a]
        dx = torch.roll(V, -1, dims=2) - V
        dx = dx + torch.roll(dx, -1, dims=1)
        dx = dx[:-1] + dx[1:]
        dy = torch.roll(V, -1, dims=1) - V
        dy = dy + torch.roll(dy, -1, dims=2)
        dy = dy[:-1] + dy[1:]
        dz = V[1:] - V[:-1]
        dz = dz + torch.roll(dz, -1, dims=2)
        dz = dz + torch.roll(dz, -1, dims=1)
        rows.append(torch.stack([dx, dy, dz]) / (4.0 * h))
    return torch.stack(rows)


def sbar_of(s):
    """sbar^2 = 1/2 sigma_0 : sigma_0 (section 3.1); s is (3, 3, ...).  Cells
    with sigma_0 = 0 get sbar = 0 without an infinite derivative."""
    tr3 = (s[0, 0] + s[1, 1] + s[2, 2]) / 3.0
    eye = torch.eye(3, dtype=s.dtype).reshape(3, 3, *([1] * (s.dim() - 2)))
    s0 = s - eye * tr3
    q = 0.5 * (s0 * s0).sum(dim=(0, 1))
    pos = q > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, q, torch.ones_like(q))),
                       torch.zeros_like(q)), s0


def dpl(p, sbar, chi):
    """Eqs. (20)-(22): D^pl = exp(-e_z/chi) exp(-Delta/T) cosh(Omega eps0 sbar /
    (k_B T)) (1 - s_Y/sbar) / tau0 above yield (and for chi > 0), else 0."""
    act = (sbar > p.sY) & (chi > 0)
    sb = torch.where(act, sbar, torch.full_like(sbar, 2.0 * p.sY))
    ch = torch.where(act, chi, torch.ones_like(chi))
    C = math.exp(-p.Delta_K / p.T) * torch.cosh(p.Omega * p.eps0 * sb / (p.kB * p.T))
    D = torch.exp(-p.ez_K / ch) * C * (1.0 - p.sY / sb) / p.tau0
    return torch.where(act, D, torch.zeros_like(D)), sb


def stress_star(v, sig, chi, h, dt, mu, p):
    """Eq. (27): sigma* = sigma + dt (L sigma + sigma L^T - tr(L) sigma
    - 2 mu D^pl sigma_0 / sbar); returns sigma*, D^pl, sbar."""
    s = _full(sig)
    L = cell_gradient(v, h)
    sb, s0 = sbar_of(s)
    D, sb_safe = dpl(p, sb, chi)
    trL = L[0, 0] + L[1, 1] + L[2, 2]
    rate = (torch.einsum("ac...,cb...->ab...", L, s) + torch.einsum("ac...,bc...->ab...", s, L)
            - trL * s - 2.0 * mu * (D / sb_safe) * s0)
    return _stored(s + dt * rate), D, sb


def chi_update(sig, chi, D, sb, h, dt, p):
    """Eq. (26): chi + (dt/c0) [(2 D^pl sbar / s_Y)(chi_inf - chi)
    + l^2 div(D^pl grad chi)], the diffusion a conservative 7-point sum with
    face coefficients (D_P + D_N)/2; the z ghost cells take sigma and chi
    extrapolated linearly from the two nearest layers and D^pl from them."""
    def ghost(k0, k1):
        sg = 2.0 * sig[:, k0] - sig[:, k1]
        cg = 2.0 * chi[k0] - chi[k1]
        sbg, _ = sbar_of(_full(sg))
        Dg, _ = dpl(p, sbg, cg)
        return cg, Dg
    ct, Dt = ghost(-1, -2)
    cb, Db = ghost(0, 1)
    chi_up = torch.cat([chi[1:], ct[None]])
    D_up = torch.cat([D[1:], Dt[None]])
    chi_dn = torch.cat([cb[None], chi[:-1]])
    D_dn = torch.cat([Db[None], D[:-1]])
    nbs = [(torch.roll(chi, s, dims=d), torch.roll(D, s, dims=d)) for d in (2, 1) for s in (-1, 1)]
    nbs += [(chi_up, D_up), (chi_dn, D_dn)]
    diff = sum(0.5 * (D + Dn) * (cn - chi) for cn, Dn in nbs)
    growth = 2.0 * D * sb / p.sY * (p.chi_inf - chi)
    return chi + dt / p.c0 * (growth + (p.l * p.l) / (h * h) * diff)


def div_rhs(ss, h, dt, mu):
    """b = (h^2/(mu dt)) div sigma* at the interior corners (planes 1..nz-1),
    the corner version of Eq. (31) over the 8 surrounding cells; zero on the
    wall planes."""
    nz, ny, nx = ss.shape[1:]
    scale = h * h / (mu * dt) / (4.0 * h)
    comps = []
    for a in range(3):
        fx, fy, fz = (ss[_COMP[a][b]] for b in range(3))
        gx = fx - torch.roll(fx, 1, dims=2)
        gx = gx + torch.roll(gx, 1, dims=1)
        gy = fy - torch.roll(fy, 1, dims=1)
        gy = gy + torch.roll(gy, 1, dims=2)
        gz = fz[1:] - fz[:-1]
        gz = gz + torch.roll(gz, 1, dims=2)
        gz = gz + torch.roll(gz, 1, dims=1)
        interior = scale * (gx[:-1] + gx[1:] + gy[:-1] + gy[1:] + gz)
        zero = torch.zeros((1, ny, nx), dtype=ss.dtype)
        comps.append(torch.cat([zero, interior, zero]))
    return torch.stack(comps)


def stress_final(v, ss, h, dt, lam, mu):
    """Eq. (29): sigma = sigma* + dt (lam tr(D) I + 2 mu D), D = sym grad v."""
    L = cell_gradient(v, h)
    D = 0.5 * (L + L.transpose(0, 1))
    trD = D[0, 0] + D[1, 1] + D[2, 2]
    eye = torch.eye(3, dtype=v.dtype).reshape(3, 3, 1, 1, 1)
    return ss + dt * _stored(lam * trD * eye + 2.0 * mu * D)


class _Solve(torch.autograd.Function):
    """v = the solution of the scaled projection system (Eq. 30) with right-
    hand side b and the wall planes of ``walls``; d v / d b is the inverse of
    the symmetric interior operator, so the backward pass is one more solve
    of the same operator with zero walls."""

    @staticmethod
    def forward(ctx, b, walls, mg, tol):
        x = walls.detach().numpy().copy()
        st, _, _ = mg.solve(b.detach().numpy().copy(), x, tol=tol, max_cycles=400)
        if st != 0:
            raise RuntimeError("oracle solve did not converge (status %d)" % st)
        ctx.mg, ctx.tol = mg, tol
        return torch.from_numpy(x)

    @staticmethod
    def backward(ctx, gv):
        g = gv.detach().numpy().copy()
        g[:, 0] = 0.0
        g[:, -1] = 0.0
        lam = g * 0.0
        if (g != 0).any():
            st, _, _ = ctx.mg.solve(g, lam, tol=ctx.tol, max_cycles=400)
            if st != 0:
                raise RuntimeError("oracle adjoint solve did not converge (status %d)" % st)
        return torch.from_numpy(lam), None, None, None


def step(mg, v, sig, chi, h, dt, lam, mu, p, bc, t, tol=1e-13):
    """One projection step (section 3.3) from t to t + dt, differentiable in
    (v, sig, chi); returns (v', sig', chi', plastic work of the step)."""
    ss, D, sb = stress_star(v, sig, chi, h, dt, mu, p)
    chi1 = chi_update(sig, chi, D, sb, h, dt, p)
    walls = v.detach().numpy().copy()
    wall_fill(walls, h, bc, t + dt)
    walls[:, 1:-1] = 0.0
    b = div_rhs(ss, h, dt, mu)
    v1 = _Solve.apply(b, torch.from_numpy(walls), mg, tol)
    sig1 = stress_final(v1, ss, h, dt, lam, mu)
    work = (2.0 * D * sb).sum() * dt * h ** 3
    return v1, sig1, chi1, work


def plastic_work(shape, v0, sig0, chi0, h, dt, lam, mu, p, bc, t0, steps, tol=1e-13):
    """W(chi^0) over ``steps`` steps from (v0, sig0, chi0) at t0, with chi0 a
    float64 tensor (set requires_grad to differentiate)."""
    mg = MG(*shape, lam, mu)
    v = torch.as_tensor(v0, dtype=_F64)
    sig = torch.as_tensor(sig0, dtype=_F64)
    chi = chi0
    W = torch.zeros((), dtype=_F64)
    t = t0
    for _ in range(steps):
        v, sig, chi, w = step(mg, v, sig, chi, h, dt, lam, mu, p, bc, t, tol)
        W = W + w
        t += dt
    return W, (v, sig, chi)


def plastic_work_gradient(shape, v0, sig0, chi0, h, dt, lam, mu, p, bc, t0, steps, tol=1e-13):
    """(W, dW/dchi^0) as (float, numpy array (nz, ny, nx))."""
    c = torch.tensor(chi0, dtype=_F64, requires_grad=True)
    W, _ = plastic_work(shape, v0, sig0, c, h, dt, lam, mu, p, bc, t0, steps, tol)
    (g,) = torch.autograd.grad(W, c)
    return float(W.detach()), g.numpy()
