"""One J/K build of a workload recipe for profilers: a warm-up build, then one build inside
an NVTX range named "jk" (ncu --nvtx --nvtx-include "jk/" selects its launches), then the
per-launch records of that build (class, team size, products path, ms, quartets).

    python -m paper_2407_09700_gb300.profile_build --workload high_l --lmin 3

--lmin keeps only the shells with l >= lmin (the f and g shells of the high-l recipe make a
build of its largest classes alone).
"""

from __future__ import annotations

import argparse

import numpy as np


def main():
    import torch

    from workloads import config_high_l, config_medium, config_scf, config_tiny, custom_molecule, random_psd_density
    from . import ERI_FP64, ERI_MIXED, Plan, build

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["tiny", "medium", "high_l", "scf"], default="medium")
    ap.add_argument("--natm", type=int, default=None)
    ap.add_argument("--lmin", type=int, default=0)
    ap.add_argument("--mixed", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    build()
    make = {"tiny": lambda: config_tiny(args.seed), "medium": lambda: config_medium(args.seed, natm=args.natm or 30),
            "high_l": lambda: config_high_l(args.seed, natm=args.natm or 12),
            "scf": lambda: config_scf(args.seed, natm=args.natm or 120)}
    m = make[args.workload]()
    if args.lmin > 0:
        shells = [(int(m.shell_atom[s]), int(m.shell_l[s]), m.exps[m.shell_off[s]:m.shell_off[s] + m.shell_nprim[s]],
                   m.coefs[m.shell_off[s]:m.shell_off[s] + m.shell_nprim[s]])
                  for s in range(m.nshell) if m.shell_l[s] >= args.lmin]
        m = custom_molecule(m.coords, shells)
        m.D = random_psd_density(m.nbf, min(40, m.nbf), np.random.default_rng(args.seed))
    plan = Plan(m, precision=ERI_MIXED if args.mixed else ERI_FP64)
    D = torch.from_numpy(np.ascontiguousarray(m.D)).cuda()
    plan.jk(D)
    torch.cuda.synchronize()
    plan.set_profiling(True)
    torch.cuda.nvtx.range_push("jk")
    plan.jk(D)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    for r in plan.launch_records():
        print(f"({r['la']}{r['lb']}|{r['lc']}{r['ld']}) team {r['team_size']} fp32 {r['fp32']} products "
              f"{r['shared_products']} compiled {r['compiled_class']} split {r['quartet_split']} listed "
              f"{r['listed']} {r['ms']:.2f} ms {r['quartets']} quartets")


if __name__ == "__main__":
    main()
