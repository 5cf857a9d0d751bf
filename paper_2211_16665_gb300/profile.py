"""One forward run with the volumetric transform on a workload, for profiler captures
(with --gradient one whole gradient of the hot path; with --td one time-domain adjoint
gradient).

    python -m paper_2211_16665_gb300.profile --workload thin_reservoir --nt 256
    python -m paper_2211_16665_gb300.profile --workload batched_towline --sources 2 --nt 128 --ring 17
    python -m paper_2211_16665_gb300.profile --workload batched_towline --sources 2 --nt 256 --gradient
    python -m paper_2211_16665_gb300.profile --workload thin_reservoir --nt 256 --td --segment 128

Runs the same kernels as a gradient's runs (H half-step with the fused
damped transform, point operators, E step), with nt limited so that a
profiler capture of a few launches ends quickly.  Not a timing tool.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="thin_reservoir")
    ap.add_argument("--nt", type=int, default=256)
    ap.add_argument("--kahan", type=int, default=1)
    ap.add_argument("--launch", default="", help="JSON keyword arguments of Engine.set_launch (skips autotuning)")
    ap.add_argument("--td", action="store_true", help="run a time-domain adjoint gradient instead")
    ap.add_argument("--segment", type=int, default=0, help="segment length of --td (0: the plan's)")
    ap.add_argument("--order", type=int, default=2, choices=[2, 4], help="spatial order of the differences")
    ap.add_argument("--sources", type=int, default=0, help="use the workload's first N sources (0: all)")
    ap.add_argument("--ring", type=int, default=0, help="cap on the E snapshot ring (csem_opts.ring_slots)")
    ap.add_argument("--gradient", action="store_true",
                    help="one whole gradient: forward with volumes, misfit against the true model's data, "
                         "adjoint-source basis, adjoint run, cell gradient")
    args = ap.parse_args()
    wl = W.ALL[args.workload]()
    if args.sources:
        wl.src = wl.src.subset(list(range(min(args.sources, wl.src.n))))
    eng = Engine.from_workload(wl, nt=args.nt, kahan=args.kahan, autotune=not args.launch, order=args.order,
                               ring_slots=args.ring)
    if args.launch:
        import json
        eng.set_launch(**json.loads(args.launch))
    rho = eng.model_tensor(wl.rho)
    if args.td:
        d = eng.fwd_model(rho, wl.src, wl.rec)
        g = eng.gradient_td(rho, wl.src, wl.rec, d, segment=args.segment)
        torch.cuda.synchronize()
        print(f"profile run ok: {wl.name}, time-domain adjoint, nt={eng.nt}, segment={eng.last_td['segment']}, "
              f"|g|max={g.abs().max().item():.3e}")
        eng.close()
        return
    if args.gradient:
        from paper_2211_16665_gb300.engine import misfit
        d_obs = eng.fwd_model(eng.model_tensor(wl.rho_true), wl.src, wl.rec)
        d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
        phi, r = misfit(d_obs, d)
        basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True, fit_target=1e-3)
        V = eng.adjoint_model(rho, wl.rec, r, basis)
        g = eng.gradient(rho, E, V)
        torch.cuda.synchronize()
        print(f"profile run ok: {wl.name}, gradient, {wl.src.n} sources, nt={eng.nt}, phi={phi.item():.3e}, "
              f"|g|max={g.abs().max().item():.3e}, launch={eng.launch_config()}")
        eng.close()
        return
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    torch.cuda.synchronize()
    print(f"profile run ok: {wl.name}, {wl.src.n} sources, nt={eng.nt}, |d|max={d.abs().max().item():.3e}, "
          f"launch={eng.launch_config()}")
    eng.close()


if __name__ == "__main__":
    main()
