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

    python -m paper_2412_16843_gb300.studies unet 64 20 1000

unet: the network first guess trained on many solver-generated pairs, as the
warm-start form asks: config-3-style 3D drops on n^3 cells (hemisphere R =
0.25, 90 deg start, theta_eq in {30, 60, 120, 150} deg, density ratio 10 or
20, viscosity ratio 10, seeded noise 1e-3), `runs` runs of `steps` steps
each; every step's last pressure solve gives one (f, rho) -> p pair (the
scaling of inputs.unet_pair), on which the network takes one Adam step as it
is generated (streamed: no pair is stored).  Then, on held-out drops of the
wide case's parameters (theta_eq = 45 deg, density ratio 20, unseen noise) at
n^3 and (2n)^3: V-cycles per solve to 1e-8 from zero, from the previous
pressure and from the network.
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


def _drop3d(n, theta_deg, ratio, seed, precision):
    from paper_2412_16843_gb300 import cdi, inputs
    h = 1.0 / n
    phi = inputs.add_noise(inputs.cap_phi_3d(n, n, n, h, 0.25, math.pi / 2, 0.5, 0.5, h), 1e-3, seed)
    rho2 = 1.0 / ratio
    s = cdi.Solver(3, (n, n, n), (1.0, 1.0, 1.0), precision)
    s.set_fluids(1.0, rho2, 0.05, 0.005, 1.0, h, 1.0)
    s.set_wall(cdi.WALL_BOTH, math.radians(theta_deg), h, 0.0)
    s.set_state(phi)
    wl = inputs.Workload("drop", 3, (n, n, n), (1.0, 1.0, 1.0), 1.0, rho2, 0.05, 0.005, 1.0, h, 1.0,
                         math.radians(theta_deg), h, 0.0, 0.0, 0.0, 1, phi)
    return s, phi, rho2, inputs.stable_dt(wl)


def unet_study(n=64, runs=20, steps=1000, eval_steps=10, tol=1e-8):
    import torch

    from paper_2412_16843_gb300 import cdi, inputs
    net = cdi.Unet((n, n, n))
    net.set_params(inputs.unet_initial_params(0))
    thetas = (30.0, 60.0, 120.0, 150.0)
    losses = []
    t0 = time.perf_counter()
    pairs = 0
    total = runs * steps
    for r in range(runs):
        theta, ratio = thetas[r % 4], (10.0, 20.0)[(r // 4) % 2]
        s, _, rho2, dt = _drop3d(n, theta, ratio, 1000 + r, cdi.FP64)
        s.set_solver(tol, 100, cdi.WARM_PREV)
        for _ in range(steps):
            s.step(dt, 1)
            f, p = s.last_pressure()
            x, t = inputs.unet_pair(f, p, s.get_fields()[0], 1.0, rho2, 1.0 / n)
            lr = 1e-3 if pairs < 0.6 * total else (3e-4 if pairs < 0.9 * total else 1e-4)
            losses.append(net.train_step(x, t, lr=lr))
            pairs += 1
        del s
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    res = {"study": "unet", "grid": n, "runs": runs, "pairs": pairs, "train_wall_s": train_s,
           "loss_first_100": float(np.mean(losses[:100])), "loss_last_1000": float(np.mean(losses[-1000:])),
           "pressure_tol": tol}
    params = net.get_params()
    del net
    for m in (n, 2 * n):
        netm = cdi.Unet((m, m, m))
        netm.set_params(params)
        ev = {}
        for name, warm in (("zero", cdi.WARM_ZERO), ("previous", cdi.WARM_PREV), ("network", cdi.WARM_UNET)):
            s, _, _, dt = _drop3d(m, 45.0, 20.0, 999, cdi.FP32_MIXED)
            s.set_exec(cdi.EXEC_KERNELS)
            s.set_solver(tol, 100, cdi.WARM_PREV)
            s.step(dt, 5)  # past the start-up solves
            s.set_solver(tol, 100, warm)
            if warm == cdi.WARM_UNET:
                s.set_warm_unet(netm)
            cyc = 0
            for _ in range(eval_steps):
                s.step(dt, 1)
                cyc += s.last_stats()["total_cycles_call"]
            ev[name] = cyc / (4.0 * eval_steps)
            del s
        res["vcycles_per_solve_%d" % m] = ev
        del netm
    return res


def main(argv):
    from paper_2412_16843_gb300 import build
    build.build()
    if len(argv) >= 2 and argv[1] == "unet":
        a = [int(v) for v in argv[2:]]
        print(json.dumps(unet_study(*a)), flush=True)
        return
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
