"""Small self-contained workloads for profiling one kernel family with ncu
(run the same command once without ncu first):

    python -m paper_2412_16843_gb300.profile_cases unet 128     # network forward passes at 128^3
    python -m paper_2412_16843_gb300.profile_cases train 64     # 3 network training steps at 64^3
    python -m paper_2412_16843_gb300.profile_cases batch 64     # 64-instance FP32-mixed sweep, 3 steps
    python -m paper_2412_16843_gb300.profile_cases drop3d 256   # 3D drop, FP32-mixed, separate kernels, 2 steps
    python -m paper_2412_16843_gb300.profile_cases wide 512 1   # 512x256x256 drop, FP32-mixed, previous-pressure
                                                                # first guess, separate kernels, 1 step
"""
import sys

import numpy as np


def main(argv):
    import torch

    from paper_2412_16843_gb300 import build, cdi, inputs
    build.build()
    mode = argv[1] if len(argv) > 1 else 'unet'
    if mode == 'unet':
        n = int(argv[2]) if len(argv) > 2 else 128
        net = cdi.Unet((n, n, n))
        net.set_params(inputs.unet_initial_params(0))
        x = torch.randn(n ** 3 * 2, dtype=torch.float32, device='cuda')
        y = torch.empty(n ** 3, dtype=torch.float32, device='cuda')
        for _ in range(3):
            net.forward_device(x, y)
        torch.cuda.synchronize()
        print('unet ok', float(y.abs().mean()))
    elif mode == 'train':
        n = int(argv[2]) if len(argv) > 2 else 64
        net = cdi.Unet((n, n, n))
        net.set_params(inputs.unet_initial_params(0))
        rng = np.random.default_rng(0)
        x = rng.standard_normal((n, n, n, 2))
        t = rng.standard_normal((n, n, n))
        for _ in range(3):
            loss = net.train_step(x, t, lr=1e-3)
        torch.cuda.synchronize()
        print('train ok', loss)
    elif mode == 'batch':
        k = int(argv[2]) if len(argv) > 2 else 64
        wls = inputs.sweep_2d(n_inst=k)
        sv = []
        for w in wls:
            s = cdi.from_workload(w, precision=cdi.FP32_MIXED, tol=1e-8)
            s.set_solver(1e-8, 100, cdi.WARM_EXTRAP)
            sv.append(s)
        b = cdi.Batch(sv)
        b.set_threads(1024)
        dts = np.array([w.dt for w in wls])
        for _ in range(3):
            b.step(dts, 1)
        torch.cuda.synchronize()
        print('batch ok', b.stats(0))
    elif mode == 'drop3d':
        n = int(argv[2]) if len(argv) > 2 else 256
        wl = inputs.drop_3d(n)
        s = cdi.from_workload(wl, precision=cdi.FP32_MIXED, tol=1e-8)
        s.set_exec(cdi.EXEC_KERNELS)
        s.step(wl.dt, 2)
        torch.cuda.synchronize()
        print('drop3d ok', s.last_stats())
    elif mode == 'wide':
        n = int(argv[2]) if len(argv) > 2 else 512
        steps = int(argv[3]) if len(argv) > 3 else 1
        wl = inputs.drop_3d_wide(n)
        s = cdi.from_workload(wl, precision=cdi.FP32_MIXED, tol=1e-8)
        s.set_exec(cdi.EXEC_KERNELS)
        s.set_solver(1e-8, 100, cdi.WARM_PREV)
        s.step(wl.dt, steps)
        torch.cuda.synchronize()
        print('wide ok', s.last_stats())


if __name__ == "__main__":
    main(sys.argv)
