"""Command line: generate one of the synthetic workloads and run it.

    python -m paper_2605_18254_gb300.run --workload poly_1m --iters 20 --precision 32

Prints the run summary (iterations, sweeps, phi, certification) as JSON.
With --iters the run stops after that many iterations of Algorithm 1 (the
profiles of single kernels use short runs); without it the RVE is generated
to its target volume fraction.  --workload platelets generates the thin
platelets of Section 3.3 (house of cards to number density 5, then
--relax sweeps with zero swelling).
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="poly_1m")
    ap.add_argument("--iters", type=int, default=0)
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--timing", action="store_true", help="per-stage CUDA event times")
    ap.add_argument("--relax", type=int, default=0, help="platelets: relaxation sweeps after the target")
    ap.add_argument("--sweep-path", type=int, default=0, choices=[0, 1, 2],
                    help="FP32 sweep kernel: 1 general path only, 2 with the staged path, 0 the default")
    ap.add_argument("--stage-capacity", type=int, default=0, help="sweep staging capacity (0: the default)")
    ap.add_argument("--plt-kernel", type=int, default=0, choices=[0, 1],
                    help="platelet sweeps and checks: 0 a block per cell where it applies, 1 warp per cell / thread per platelet")
    a = ap.parse_args(argv)
    import torch

    import srm_inputs
    import paper_2605_18254_gb300 as srm

    if a.workload == "platelets":
        return run_platelets(a, srm, srm_inputs, torch)
    w = srm_inputs.RECIPES[a.workload]()
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x,
                precision=a.precision, c_m=w.c_m, c_w=w.c_w, N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake)
    if a.sweep_path or a.stage_capacity:
        g.set_tuning(0, a.stage_capacity, a.sweep_path)
    if a.timing:
        g.set_timing(True)
    t0 = time.perf_counter()
    info = g.run_to_target(a.iters if a.iters > 0 else 1 << 40)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    pairs, gap, phi = g.certify()
    out = dict(workload=w.name, n=w.n, precision=a.precision, wall_s=wall, **info,
               certified_pairs=pairs, min_gap=gap, state=g.state(), tuning=g.tuning())
    if a.timing:
        out["timings"] = g.timings()
    g.close()
    print(json.dumps(out, default=float))


def run_platelets(a, srm, srm_inputs, torch):
    w = srm_inputs.platelets()
    g = srm.Platelets(w.box, w.x, w.u, w.a0, w.t0, w.lambda0, 1.0, w.seed, c_w=w.c_w, c_m=w.c_m, c_r=w.c_r,
                      sweep_kernel=a.plt_kernel)
    t0 = time.perf_counter()
    info = g.run_to_target(a.iters if a.iters > 0 else 0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    relaxed = 0
    if a.relax > 0:
        g.set_params(c_w=0.0, c_m=0.1 * w.extra["D"], c_r=0.1)
        relaxed = g.sweeps(a.relax)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    cnt, _ = g.check()
    _, _, st = g.state()
    stats = g.sweep_stats()
    g.close()
    print(json.dumps(dict(workload="platelets", n=w.n, generation_s=t1 - t0, relax_s=t2 - t1,
                          relax_sweeps=a.relax, relax_moves=relaxed, colliding=cnt, **info, state=st,
                          sweep_stats=stats),
                     default=float))


if __name__ == "__main__":
    main()
