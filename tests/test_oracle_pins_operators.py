"""Pins of the oracle's momentum operator and of every slip model against
closed forms the mathematics fixes.

* The viscous term of Eq. (NS_momentum), div[mu (grad u + grad u^T)], with mu
  varying in space (mu linear in phi, Sec. 2) and velocity fields whose every
  cross derivative is nonzero: the discrete operator must converge at second
  order to the closed form written out below, in 2D and 3D.  The advection
  term -div(rho u x u) (mass flux m = rho_f u when gamma = 0) is pinned the
  same way.  With sigma = gamma = 0 the right-hand side is R(u) = A(u) + V(u)
  with A quadratic and V linear in u, so R(u) and R(2u) give both parts
  exactly: V = 2 R(u) - R(2u)/2 and A = (R(2u) - 2 R(u))/2.
* Every slip model of Sec. 3 (Eqs. Model 1A .. Model 4B) on a planar
  interface: at theta = theta_eq the model's bracket vanishes (to round-off for
  the psi models, whose psi is exactly linear; at second order for the phi
  models, whose discrete phi derivatives carry O(h^2) errors), and the wall
  integral of u^Y converges at second order to the value that Eq. (integral
  constraint u_slip) fixes, -(sigma/beta)(cos theta - cos theta_eq) for a
  right contact line with tau = +x.
  On a 3D wall the slip is a tangential vector: with the contact line oblique to
  the grid (in-wall normal along (1, 2)) each tangential component, summed
  along a grid line that crosses the contact line, must converge to the same
  constraint value (the line element along the normal is cos or sin of the
  direction times h), which pins the second tangential component, the
  direction of the slip vector and the tangential gradient inside |grad psi|.
  A planar profile wider than eps (|grad psi| != 1, kappa != 0) separates
  the |grad psi| forms (B) from the equilibrium forms (A) and pins the
  curvature correction of Models 3 and 4 by a closed-form integral.
* The surface tension force of Eq. (EB surface tension) with the chemical
  potential of Eq. (chemical potential), against its closed form for a
  smooth phi.
* The wall-row one-sided stencils of Sec. 4 on polynomial psi: the
  first-derivative stencil is exact for quadratics, the second-derivative
  stencil for cubics.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2412_16843_gb300 import inputs

INF = float("inf")


class Sep:
    """c * prod_b sin(k_b x_b + a_b): every partial derivative in closed form,
    d^n/dx^n sin(kx + a) = k^n sin(kx + a + n pi/2)."""

    def __init__(self, c, k, a):
        self.c, self.k, self.a = c, k, a

    def __call__(self, X, orders=(0, 0, 0)):
        out = self.c
        for b, x in enumerate(X):
            o = orders[b]
            out = out * self.k[b] ** o * np.sin(self.k[b] * x + self.a[b] + o * math.pi / 2)
        return out


def d(f, X, *axes):
    """Partial derivative of a Sep along the listed axes."""
    o = [0, 0, 0]
    for b in axes:
        o[b] += 1
    return f(X, tuple(o))


def face_coords(n, h, a, dim):
    """Coordinates of the faces of component a, shaped like the face array
    (the low face of cell q sits at q_a h along a, cell centres elsewhere)."""
    shape = list(n)
    if a == dim - 1:
        shape[a] += 1
    axes = []
    for b in range(dim):
        idx = np.arange(shape[b], dtype=np.float64)
        axes.append(idx * h if b == a else (idx + 0.5) * h)
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return [grids[dim - 1 - b] for b in range(dim)]


def cell_coords(n, h, dim):
    axes = [(np.arange(n[b], dtype=np.float64) + 0.5) * h for b in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return [grids[dim - 1 - b] for b in range(dim)]


def fields(dim, L):
    """phi (smooth, inside (0.2, 0.8)) and a velocity field with nonzero
    divergence and every cross derivative nonzero; periodic along the
    periodic axes."""
    kx = 2 * math.pi / L[0]
    if dim == 2:
        q = 1.3 * math.pi / L[1]
        phi = Sep(0.3, (kx, q, 0.0), (0.4, 0.9, math.pi / 2))
        vel = [Sep(0.8, (kx, q, 0.0), (0.2, 0.5, math.pi / 2)),
               Sep(0.6, (2 * kx, 0.7 * q, 0.0), (1.1, 0.3, math.pi / 2))]
    else:
        ky = 2 * math.pi / L[1]
        q = 1.3 * math.pi / L[2]
        phi = Sep(0.3, (kx, ky, q), (0.4, 0.7, 0.9))
        vel = [Sep(0.8, (kx, ky, q), (0.2, 1.0, 0.5)),
               Sep(0.6, (2 * kx, ky, 0.7 * q), (1.1, 0.4, 0.3)),
               Sep(0.5, (kx, 2 * ky, q), (0.6, 0.8, 1.2))]
    return phi, vel


def closed_forms(dim, X, a, phi, vel, mu_c, rho_c):
    """Closed forms at the points X of component a's faces:
    visc_a = sum_b d_b[mu (d_b u_a + d_a u_b)]
           = sum_b [mu_b (d_b u_a + d_a u_b) + mu (d_bb u_a + d_ab u_b)],
    adv_a  = -sum_b d_b(rho u_b u_a)
           = -sum_b [rho_b u_b u_a + rho (d_b u_b u_a + u_b d_b u_a)],
    with mu = mu2 + dmu (0.5 + phi'), rho likewise (phi = 0.5 + phi')."""
    mu2, dmu = mu_c
    rho2, drho = rho_c
    ph = 0.5 + phi(X)
    mu = mu2 + dmu * ph
    rho = rho2 + drho * ph
    ua = vel[a](X)
    visc = np.zeros_like(ua)
    adv = np.zeros_like(ua)
    for b in range(dim):
        mub = dmu * d(phi, X, b)
        rhob = drho * d(phi, X, b)
        ub = vel[b](X)
        visc += mub * (d(vel[a], X, b) + d(vel[b], X, a)) + mu * (d(vel[a], X, b, b) + d(vel[b], X, a, b))
        adv -= rhob * ub * ua + rho * (d(vel[b], X, b) * ua + ub * d(vel[a], X, b))
    return visc, adv


def split_rhs(dim, n, L, mu_c, rho_c):
    """Discrete viscous and advective parts of the momentum right-hand side
    (2 R(u) - R(2u)/2 and (R(2u) - 2 R(u))/2), and the closed forms on the same
    faces."""
    h = L[0] / n[0]
    o = oracle.Oracle(dim, n, L)
    mu2, dmu = mu_c
    rho2, drho = rho_c
    # mu_i, rho_i of the two fluids; sigma = 0, gamma = 0, no-slip walls (the
    # ghost value is then -u_0: linear in u)
    o.set_fluids(rho2 + drho, rho2, mu2 + dmu, mu2, 0.0, h, 0.0)
    o.set_wall(2, math.pi / 2, INF, INF)
    phi, vel = fields(dim, L)
    Xc = cell_coords(n, h, dim)
    phic = 0.5 + phi(Xc)
    vf = [vel[a](face_coords(n, h, a, dim)) for a in range(dim)]
    vf[dim - 1][0] = 0.0       # wall faces carry no normal velocity
    vf[dim - 1][-1] = 0.0
    o.set_state(phic, vf)
    _, r1 = o.eval_rhs(gamma=0.0)
    o.set_state(phic, [2.0 * v for v in vf])
    _, r2 = o.eval_rhs(gamma=0.0)
    out = []
    for a in range(dim):
        V = 2.0 * r1[a] - 0.5 * r2[a]
        A = 0.5 * (r2[a] - 2.0 * r1[a])
        X = face_coords(n, h, a, dim)
        visc, adv = closed_forms(dim, X, a, phi, vel, mu_c, rho_c)
        # compare on the same physical region at every resolution, away from
        # the walls (the wall rows take the ghost value, which these fields
        # do not satisfy): the middle 60 % of the wall axis
        W = dim - 1
        LW = n[W] * h
        idx = (X[W] >= 0.2 * LW) & (X[W] <= 0.8 * LW)
        out.append((V[idx], visc[idx], A[idx], adv[idx]))
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_viscous_operator_variable_mu_converges_to_closed_form(dim):
    """Eq. (NS_momentum): div[mu(grad u + grad u^T)] with mu linear in phi
    (Sec. 2).  Every component's discrete viscous term converges at second
    order to the closed form.  A dropped grad u^T term, a normal-stress factor
    mu instead of 2 mu, or a misplaced edge viscosity would leave an O(1)
    error here (the fields have nonzero divergence and nonzero cross
    derivatives, and mu varies)."""
    mu_c = (0.1, 0.2)      # mu2, mu1 - mu2
    rho_c = (1.0, 1.5)     # rho2, rho1 - rho2
    sizes = (32, 64, 128) if dim == 2 else (16, 32, 64)
    errs = {a: [] for a in range(dim)}
    scale = None
    for nx in sizes:
        if dim == 2:
            n, L = (nx, nx // 2), (1.0, 0.5)
        else:
            n, L = (nx, nx, nx // 2), (1.0, 1.0, 0.5)
        parts = split_rhs(dim, n, L, mu_c, rho_c)
        for a, (V, visc, _, _) in enumerate(parts):
            if scale is None:
                scale = np.abs(visc).max()
            errs[a].append(np.abs(V - visc).max() / scale)
    for a in range(dim):
        e = errs[a]
        assert e[-1] < 0.02, (a, e)
        assert e[0] / e[1] > 3.3 and e[1] / e[2] > 3.5, (a, e)


@pytest.mark.parametrize("dim", [2, 3])
def test_advection_operator_converges_to_closed_form(dim):
    """Eq. (NS_momentum) advection -div(rho u x u) with the consistent mass
    flux m = (rho1 - rho2) u phi_f + rho2 u_f = rho_f u_f (gamma = 0):
    second-order convergence to the closed form for every component."""
    mu_c = (0.1, 0.2)
    rho_c = (1.0, 1.5)
    sizes = (32, 64, 128) if dim == 2 else (16, 32, 64)
    errs = {a: [] for a in range(dim)}
    scale = None
    for nx in sizes:
        if dim == 2:
            n, L = (nx, nx // 2), (1.0, 0.5)
        else:
            n, L = (nx, nx, nx // 2), (1.0, 1.0, 0.5)
        parts = split_rhs(dim, n, L, mu_c, rho_c)
        for a, (_, _, A, adv) in enumerate(parts):
            if scale is None:
                scale = np.abs(adv).max()
            errs[a].append(np.abs(A - adv).max() / scale)
    for a in range(dim):
        e = errs[a]
        assert e[-1] < 0.02, (a, e)
        assert e[0] / e[1] > 3.3 and e[1] / e[2] > 3.5, (a, e)


# ---------------------------------------------------------------------------
# slip models on a planar interface
# ---------------------------------------------------------------------------

MODELS = ["1A", "1B", "2A", "2B", "3A", "3B", "4A", "4B"]
PSI_MODELS = {"2A", "2B", "4A", "4B"}


def _tilted(nx, ny, h, x0, theta, eps):
    """Planar interface through (x0, 0) at contact angle theta (fluid 1 on the
    left), with a parallel interface half a period away so the field is
    periodic in x."""
    x = inputs.cell_centres(nx, h)[None, :]
    y = inputs.cell_centres(ny, h)[:, None]
    nu = (-math.sin(theta), -math.cos(theta))
    dd = nu[0] * (x - x0) + nu[1] * y
    phi_r = 0.5 * (1 + np.tanh(dd / (2 * eps)))
    d2 = -nu[0] * (x - (x0 - 0.5 * nx * h)) - nu[1] * y
    phi_l = 0.5 * (1 + np.tanh(d2 / (2 * eps)))
    return phi_r + phi_l - 1.0


def _slip(model, nx, ny, Lx, th, th_eq, eps, sigma=1.0, beta=10.0, x0=1.4):
    h = Lx / nx
    o = oracle.Oracle(2, (nx, ny), (Lx, ny * h))
    o.set_fluids(1.0, 1.0, 0.1, 0.1, sigma, eps, 1.0)
    o.set_wall(2, th_eq, beta, beta)
    o.set_model(model)
    o.set_state(_tilted(nx, ny, h, x0, th, eps))
    uY, _, _ = o.eval_wall()
    x = np.arange(nx) * h      # u-face positions on the wall
    return uY[0, 0], x, h


@pytest.mark.parametrize("model", MODELS)
def test_slip_model_vanishes_at_equilibrium_angle_planar(model):
    """Eqs. (Model 1A .. 4B) at theta = theta_eq on a planar interface (kappa = 0,
    psi linear, eps grad phi = phi(1-phi) n): the bracket A + B cos(theta_eq) is
    zero in the continuum for every model.  Psi models: psi is exactly linear,
    so u^Y = 0 to round-off.  Phi models: their phi differences carry O(h^2)
    errors, so max |u^Y| falls at second order."""
    th = math.radians(55.0)
    sigma, beta = 1.0, 10.0
    eps = 0.03
    scale = 6 * sigma / beta * 0.0625 / eps     # (6 sigma/beta) P_max^2 |d_tau psi|/eps
    vals = []
    for nx in (128, 256, 512):
        uY, x, h = _slip(model, nx, nx // 8, 2.0, th, th, eps, sigma, beta)
        win = np.abs(x - 1.4) < 0.3
        vals.append(np.abs(uY[win]).max() / scale)
    if model in PSI_MODELS:
        assert max(vals) < 1e-10, vals
    else:
        assert vals[0] / vals[1] > 3.3 and vals[1] / vals[2] > 3.6, vals
        assert vals[-1] < 2e-3, vals


@pytest.mark.parametrize("model", MODELS)
def test_slip_model_integral_constraint_planar(model):
    """Eq. (integral constraint u_slip), which the paper states every model
    satisfies: on a planar interface at theta != theta_eq the wall integral of
    u^Y is -(sigma/beta)(cos theta - cos theta_eq) for a right contact line
    (tau = +x).  The discrete sum converges to it at second order with eps
    fixed."""
    th, th_eq = math.radians(70.0), math.radians(50.0)
    sigma, beta, eps = 1.0, 10.0, 0.02
    exact = -(sigma / beta) * (math.cos(th) - math.cos(th_eq))
    errs = []
    for nx in (256, 512, 1024):
        uY, x, h = _slip(model, nx, nx // 16, 2.0, th, th_eq, eps, sigma, beta)
        win = np.abs(x - 1.4) < 0.3
        errs.append(abs(uY[win].sum() * h - exact) / abs(exact))
    assert errs[-1] < 5e-3, errs
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.5, errs


@pytest.mark.parametrize("model", MODELS)
def test_slip_model_vanishes_at_equilibrium_angle_high_wall(model):
    """The high wall (inward normal -y) of the same planar interfaces: the
    lines cross the channel, so fluid 1 meets the high wall at pi - theta.
    With theta_eq = pi - theta there, the bracket of every model vanishes as on
    the low wall (psi models to round-off, here 1e-9 of the slip scale because
    the mirrored line's tails reach the high wall's window; phi models at
    second order), which pins the sign of the one-sided normal derivatives of
    the high wall."""
    th = math.radians(55.0)
    sigma, beta, eps = 1.0, 10.0, 0.03
    scale = 6 * sigma / beta * 0.0625 / eps
    vals = []
    for nx in (128, 256, 512):
        h = 2.0 / nx
        ny = nx // 8
        o = oracle.Oracle(2, (nx, ny), (2.0, ny * h))
        o.set_fluids(1.0, 1.0, 0.1, 0.1, sigma, eps, 1.0)
        o.set_wall(0, th, beta, beta)
        o.set_wall(1, math.pi - th, beta, beta)
        o.set_model(model)
        o.set_state(_tilted(nx, ny, h, 1.4, th, eps))
        uY, _, _ = o.eval_wall()
        x = np.arange(nx) * h
        xt = 1.4 - ny * h / math.tan(th)      # where the right line meets the high wall
        win = np.abs(x - xt) < 0.3
        vals.append(np.abs(uY[1, 0][win]).max() / scale)
    if model in PSI_MODELS:
        assert max(vals) < 1e-9, vals
    else:
        assert vals[0] / vals[1] > 3.3 and vals[1] / vals[2] > 3.6, vals
        assert vals[-1] < 2e-3, vals


def test_wall_curvature_extrapolation_second_order():
    """Reading R4: kappa_p (= kappa in 2D, Eq. curvature) is extrapolated to
    the wall linearly from the first two cell rows.  For a circle crossing the
    wall, psi = R - r and kappa = 1/r in the continuum, so with eps fixed the
    wall value at each column near the contact line converges to 1/r at the
    wall point at second order (a copy of the first row would be first order)."""
    R, yc, eps = 0.3, -0.1, 0.03
    errs = []
    for nx in (128, 256, 512):
        h = 1.0 / nx
        ny = nx // 2
        o = oracle.Oracle(2, (nx, ny), (1.0, ny * h))
        o.set_fluids(1.0, 1.0, 0.1, 0.1, 1.0, eps, 1.0)
        o.set_wall(2, math.pi / 2, 10.0, 10.0)
        x = inputs.cell_centres(nx, h)
        y = inputs.cell_centres(ny, h)
        X, Y = np.meshgrid(x, y)
        r = np.sqrt((X - 0.5) ** 2 + (Y - yc) ** 2)
        o.set_state(0.5 * (1 + np.tanh((R - r) / (2 * eps))))
        _, kpw = o.wall_columns()
        rw = np.sqrt((x - 0.5) ** 2 + yc ** 2)
        near = np.abs(rw - R) < 2 * eps
        errs.append(np.abs(kpw[0][near] - 1 / rw[near]).max())
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.5, errs


def _oblique_3d(nx, ny, nz, h, theta, eps, a, b, s0):
    """3D planar interface at contact angle theta on the low wall whose contact
    line is sigma = s0, sigma = (a x + b y)/|(a, b)| (fluid 1 on the side of
    smaller sigma), and a mirrored interface half a period of sigma away, so
    the field is periodic in x and y (a Lx = b Ly is the period of a x + b y)."""
    x = inputs.cell_centres(nx, h)[None, None, :]
    y = inputs.cell_centres(ny, h)[None, :, None]
    z = inputs.cell_centres(nz, h)[:, None, None]
    c = math.hypot(a, b)
    P = nx * h * a / c
    v = ((a * x + b * y) / c - s0 + P / 4) % P - P / 4   # right line at v = 0, left one at v = P/2
    pr = 0.5 * (1 + np.tanh((-math.sin(theta) * v - math.cos(theta) * z) / (2 * eps)))
    pl = 0.5 * (1 + np.tanh((math.sin(theta) * (v - P / 2) - math.cos(theta) * z) / (2 * eps)))
    return pr + pl, P


@pytest.mark.parametrize("model", ["1A", "1B", "3A", "3B"])
def test_phi_slip_models_vanish_at_equilibrium_angle_oblique_3d(model):
    """The phi models on the oblique 3D wall at theta = theta_eq = 55 deg:
    their bracket vanishes in the continuum, and the discrete slip (both
    tangential components, at every face near the right contact line) falls
    at second order with eps fixed.  Their |grad phi| takes the other
    tangential phi gradient extrapolated linearly to the wall; a copy of the
    first row would leave a first-order error."""
    th = math.radians(55.0)
    sigma, beta, eps, L, a, b, nz = 1.0, 10.0, 0.05, 4.0, 1, 2, 8
    c = math.hypot(a, b)
    vals = []
    for nx in (256, 512):
        h = L / nx
        ny = nx * a // b
        o = oracle.Oracle(3, (nx, ny, nz), (L, ny * h, nz * h))
        o.set_fluids(1.0, 1.0, 0.1, 0.1, sigma, eps, 1.0)
        o.set_wall(2, th, beta, beta)
        o.set_model(model)
        s0 = 0.6 * L * a / c
        phi, P = _oblique_3d(nx, ny, nz, h, th, eps, a, b, s0)
        o.set_state(phi)
        uY, _, _ = o.eval_wall()
        wrap = lambda d: (d + P / 2) % P - P / 2
        sx = (a * np.arange(nx)[None, :] * h + b * inputs.cell_centres(ny, h)[:, None]) / c
        sy = (a * inputs.cell_centres(nx, h)[None, :] + b * np.arange(ny)[:, None] * h) / c
        vals.append(max(np.abs(uY[0, 0][np.abs(wrap(sx - s0)) < P / 4]).max(),
                        np.abs(uY[0, 1][np.abs(wrap(sy - s0)) < P / 4]).max()))
    assert vals[0] / vals[1] > 3.3 and vals[1] < 1.5e-3, vals


@pytest.mark.parametrize("model", MODELS)
def test_slip_model_integral_constraint_oblique_3d(model):
    """Eq. (integral constraint u_slip) on a 3D wall with the contact line
    oblique to the grid (in-wall normal (1, 2)/sqrt 5, theta = 70 deg,
    theta_eq = 50 deg, eps fixed): in every grid row the sum of the x component
    of u^Y times h over the right contact line, and in every grid column the
    sum of the y component, converge at second order to
    -(sigma/beta)(cos theta - cos theta_eq)."""
    th, th_eq = math.radians(70.0), math.radians(50.0)
    sigma, beta, eps, L, a, b, nz = 1.0, 10.0, 0.05, 4.0, 1, 2, 8
    exact = -(sigma / beta) * (math.cos(th) - math.cos(th_eq))
    c = math.hypot(a, b)
    errs = []
    for nx in (256, 512):
        h = L / nx
        ny = nx * a // b
        o = oracle.Oracle(3, (nx, ny, nz), (L, ny * h, nz * h))
        o.set_fluids(1.0, 1.0, 0.1, 0.1, sigma, eps, 1.0)
        o.set_wall(2, th_eq, beta, beta)
        o.set_model(model)
        s0 = 0.6 * L * a / c
        phi, P = _oblique_3d(nx, ny, nz, h, th, eps, a, b, s0)
        o.set_state(phi)
        uY, _, _ = o.eval_wall()
        wrap = lambda d: (d + P / 2) % P - P / 2
        # x component on x faces (x = i h, cell-centre y), y component on y faces
        sx = (a * np.arange(nx)[None, :] * h + b * inputs.cell_centres(ny, h)[:, None]) / c
        sy = (a * inputs.cell_centres(nx, h)[None, :] + b * np.arange(ny)[:, None] * h) / c
        Ix = (uY[0, 0] * (np.abs(wrap(sx - s0)) < P / 4)).sum(axis=1) * h
        Iy = (uY[0, 1] * (np.abs(wrap(sy - s0)) < P / 4)).sum(axis=0) * h
        errs.append((np.abs(Ix - exact).max() / abs(exact), np.abs(Iy - exact).max() / abs(exact)))
    for comp in range(2):
        assert errs[-1][comp] < 1.5e-3, errs
        assert errs[0][comp] / errs[1][comp] > 3.3, errs


@pytest.mark.parametrize("model", MODELS)
def test_slip_models_on_profile_thicker_than_eps(model):
    """The same planar interface with a tanh profile of width eps' = eps/r
    (r = 0.8), i.e. away from the phase-field equilibrium: psi = r d,
    |grad psi| = r, and Eq. (curvature) gives kappa = (1-2 phi)(1-r^2)/eps.
    Integrating each model of Sec. 3 across the contact line in closed form
    (P = phi(1-phi) = sech^2(s/2)/4 with s = d/eps'; int P^2 dtau =
    eps'/(6 |d_tau d|); int P^2 (1-2 phi) s ds = -1/12):
      A models (1A, 2A):  -(sigma/beta)(r cos theta - cos theta_eq),
      B models (1B, 2B):  -(sigma/beta) r (cos theta - cos theta_eq),
      with the curvature correction (1 + kappa_p psi) of 3A/4A (3B/4B) an
      extra -(sigma/(2 beta)) b (1 - r^2) cos theta_eq, b = 1 (b = r).
    The discrete wall sums converge to these at second order, which separates
    the |grad| forms from the equilibrium forms and pins the correction."""
    th, th_eq = math.radians(70.0), math.radians(50.0)
    sigma, beta, eps, r = 1.0, 10.0, 0.02, 0.8
    b = r if model.endswith("B") else 1.0
    exact = -(sigma / beta) * (r * math.cos(th) - math.cos(th_eq)) if b == 1.0 else \
        -(sigma / beta) * r * (math.cos(th) - math.cos(th_eq))
    if model[0] in "34":
        exact -= sigma / (2 * beta) * b * (1 - r * r) * math.cos(th_eq)
    errs = []
    for nx in (256, 512, 1024):
        ny = nx // 16
        h = 2.0 / nx
        o = oracle.Oracle(2, (nx, ny), (2.0, ny * h))
        o.set_fluids(1.0, 1.0, 0.1, 0.1, sigma, eps, 1.0)
        o.set_wall(2, th_eq, beta, beta)
        o.set_model(model)
        o.set_state(_tilted(nx, ny, h, 1.4, th, eps / r))
        uY, _, _ = o.eval_wall()
        x = np.arange(nx) * h
        win = np.abs(x - 1.4) < 0.35
        errs.append(abs(uY[0, 0, win].sum() * h - exact) / abs(exact))
    assert errs[-1] < 5e-4, errs
    assert errs[0] / errs[1] > 3.6 and errs[1] / errs[2] > 3.8, errs


# ---------------------------------------------------------------------------
# surface tension force (Eq. EB surface tension with Eq. chemical potential)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_surface_tension_force_converges_to_closed_form(dim):
    """With u = 0 the momentum right-hand side is the surface tension force
    alone, F_ST = mu_c grad phi (Eq. EB surface tension).  For a smooth phi,
    psi = eps ln(phi/(1-phi)) has grad psi = eps grad phi / P and
    lap psi = eps [lap phi / P - (1-2 phi)|grad phi|^2 / P^2] (P = phi(1-phi),
    dP/dphi = 1-2 phi), so Eq. (chemical potential) is
    mu_c = 6 sigma [P (1-2 phi)(1 - |grad psi|^2)/eps - P lap psi] in closed
    form.  The discrete face force converges to mu_c d_a phi at second order."""
    sigma, eps = 0.7, 0.05
    errs = {a: [] for a in range(dim)}
    scale = None
    for nx in ((32, 64, 128) if dim == 2 else (24, 48, 96)):
        if dim == 2:
            n, L = (nx, nx // 2), (1.0, 0.5)
        else:
            n, L = (nx, nx, nx // 2), (1.0, 1.0, 0.5)
        h = L[0] / n[0]
        phi, _ = fields(dim, L)
        o = oracle.Oracle(dim, n, L)
        o.set_fluids(1.3, 1.0, 0.1, 0.05, sigma, eps, 1.0)
        o.set_wall(2, math.radians(60.0), 5.0, 5.0)
        o.set_state(0.5 + phi(cell_coords(n, h, dim)))
        _, rm = o.eval_rhs(gamma=1.0)
        for a in range(dim):
            X = face_coords(n, h, a, dim)
            ph = 0.5 + phi(X)
            P = ph * (1 - ph)
            g2 = sum(d(phi, X, b) ** 2 for b in range(dim))
            lap_phi = sum(d(phi, X, b, b) for b in range(dim))
            gpsi2 = eps * eps * g2 / P ** 2
            lap_psi = eps * (lap_phi / P - (1 - 2 * ph) * g2 / P ** 2)
            muc = 6 * sigma * (P * (1 - 2 * ph) * (1 - gpsi2) / eps - P * lap_psi)
            F = muc * d(phi, X, a)
            W = dim - 1
            LW = n[W] * h
            keep = (X[W] >= 0.2 * LW) & (X[W] <= 0.8 * LW)
            if scale is None:
                scale = np.abs(F[keep]).max()
            errs[a].append(np.abs(rm[a][keep] - F[keep]).max() / scale)
    for a in range(dim):
        e = errs[a]
        assert e[-1] < 0.02, (a, e)
        assert e[0] / e[1] > 3.3 and e[1] / e[2] > 3.5, (a, e)


# ---------------------------------------------------------------------------
# wall-row one-sided stencils on polynomials
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("degree", [2, 3])
def test_wall_row_stencils_exact_on_polynomials(degree):
    """Sec. 4: second-order one-sided wall-normal stencils in the first and
    last cell rows.  For psi a polynomial in y: the first derivative (one-sided
    and central) is exact for a quadratic; the second derivative (one-sided
    four-point and central three-point) is exact for a cubic.  The phase field
    is built from psi through the inverse of Eq. (psi), phi = 1/(1 + e^(-psi/eps))."""
    nx, ny = 8, 16
    h = 1.0 / nx
    eps = 1.0
    o = oracle.Oracle(2, (nx, ny), (1.0, ny * h))
    o.set_fluids(1, 1, 0.1, 0.1, 1.0, eps, 0.0)
    y = inputs.cell_centres(ny, h)
    c = (0.3, -1.2, 0.9, 0.2 if degree == 3 else 0.0)
    psi = c[0] + c[1] * y + c[2] * y ** 2 + c[3] * y ** 3
    dpsi = c[1] + 2 * c[2] * y + 3 * c[3] * y ** 2
    d2psi = 2 * c[2] + 6 * c[3] * y
    phi = np.repeat((1.0 / (1.0 + np.exp(-psi / eps)))[:, None], nx, axis=1)
    out = o.eval_psi(phi)
    assert np.abs(out["psi"] - psi[:, None]).max() < 1e-13
    assert np.abs(out["lap"] - d2psi[:, None]).max() < 1e-10
    if degree == 2:
        assert np.abs(out["gy"] - dpsi[:, None]).max() < 1e-11
    assert np.abs(out["gx"]).max() < 1e-13
