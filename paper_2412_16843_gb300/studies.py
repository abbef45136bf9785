"""Long runs of the paper's own cases through the C ABI (results quoted in
the design notes; each prints one JSON line per run):

    python -m paper_2412_16843_gb300.studies f3 32 64 128

f3: the equilibrium drop of Sec. 5.1 (a half disc of radius 0.15 on the wall
of [0,1] x [0,0.5], 90 deg start, theta_eq = 60 deg, rho = mu = 0.01 in both
fluids, sigma = 1, beta = 10, gamma = 2.5 |u|_max, Model 4A, FP64) on the
mesh family of Figs. 9 and 10, eps ~ h^(2/3) (1.4 h at 64 cells across).
Each mesh runs until its wetted length changes by less than 1e-6 relative
over 0.1 time units (at most t_max): then the maximum slip velocity along the
wall, max |u_w - U| with u_w the wall value of the tangential velocity
(mean of the first row and its ghost value), and the relative wetted-length
error L_err = (L - L_exact) / L_exact, L_exact = 2 R_eq sin(theta_eq) of the
cap with the initial area.  The paper reports max |u_slip| ~ N_x^(-1/2) and
L_err ~ N_x^(-1).
"""
import json
import math
import sys
import time

import numpy as np


def f3_run(nx, t_max=6.0, window=0.1, rtol=1e-6):
    import torch

    from paper_2412_16843_gb300 import cdi, inputs
    Lx, R0, rho, mu, sigma, beta = 1.0, 0.15, 0.01, 0.01, 1.0, 10.0
    th0, th_eq = math.pi / 2, math.radians(60.0)
    ny = nx // 2
    h = Lx / nx
    eps = 1.4 * (1.0 / 64) * (h * 64) ** (2.0 / 3.0)
    R = inputs.cap_radius(R0, th0)
    phi = inputs.cap_phi_2d(nx, ny, h, R, th0, 0.5, eps)
    s = cdi.Solver(2, (nx, ny), (Lx, ny * h))
    s.set_fluids(rho, rho, mu, mu, sigma, eps, -0.01)
    s.set_wall(cdi.WALL_BOTH, th_eq, 0.01)
    s.set_wall_beta(cdi.WALL_BOTH, beta, beta)
    s.set_solver(1e-10, 100, cdi.WARM_EXTRAP)
    s.set_exec(cdi.EXEC_PERSISTENT)
    s.set_phi(phi)
    m0 = s.mass()
    wl = inputs.Workload("drop", 2, (nx, ny), (Lx, ny * h), rho, rho, mu, mu, sigma, eps, 0.0, th_eq, 0.0,
                         0.0, 0.0, 0.0, 1, phi)
    dt = inputs.stable_dt(wl, 0.35)
    chunk = max(1, int(round(window / dt)))
    dt = window / chunk
    R_eq = inputs.cap_radius(R0, th_eq)
    L_exact = 2.0 * R_eq * math.sin(th_eq)
    t, L_prev, steady = 0.0, None, False
    t0 = time.perf_counter()
    while t < t_max - 1e-12:
        s.step(dt, chunk)
        t += window
        _, L = s.contact_angle(0)
        if L_prev is not None and abs(L - L_prev) <= rtol * L:
            steady = True
            break
        L_prev = L
    torch.cuda.synchronize()
    th, L = s.contact_angle(0)
    _, vel, _ = s.get_fields()
    _, ghost = s.eval_wall()
    u_w = 0.5 * (vel[0][0] + ghost[0, 0])          # low wall: first row and its ghost value
    return {"study": "f3", "nx": nx, "eps_over_h": eps / h, "dt": dt, "t": t, "steady": steady,
            "steps": int(round(t / dt)), "wall_s": time.perf_counter() - t0,
            "theta_deg": math.degrees(th), "L": L, "L_exact": L_exact, "L_err": (L - L_exact) / L_exact,
            "max_u_slip": float(np.abs(u_w).max()), "mass_drift": abs(s.mass() - m0) / m0}


def main(argv):
    from paper_2412_16843_gb300 import build
    build.build()
    if len(argv) < 2 or argv[1] != "f3":
        raise SystemExit(__doc__)
    sizes = [int(a) for a in argv[2:]] or [32, 64, 128]
    res = []
    for n in sizes:
        r = f3_run(n)
        res.append(r)
        print(json.dumps(r), flush=True)
    if len(res) >= 2:
        n = np.log([r["nx"] for r in res])
        for key in ("max_u_slip", "L_err"):
            v = np.log(np.abs([r[key] for r in res]))
            slope = float(np.polyfit(n, v, 1)[0])
            pair = [float((v[i + 1] - v[i]) / (n[i + 1] - n[i])) for i in range(len(res) - 1)]
            print(json.dumps({"study": "f3", "fit": key, "slope": slope, "pairwise": pair}), flush=True)


if __name__ == "__main__":
    main(sys.argv)
