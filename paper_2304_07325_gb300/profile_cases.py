"""Small, self-contained workloads for profiling single kernels (ncu, CUDA events).

    python -m paper_2304_07325_gb300.profile_cases step --n 10000 [--precision mixed] [--n-field F]
        one step of the Sec. 3 disk (plus F field particles); the trapezoid kicks (k_trap_*) and,
        with field particles, the field rectangle (k_field_*) run twice
    python -m paper_2304_07325_gb300.profile_cases bound_pair [--steps 1]
        one step of a 5-body encounter group of the 10,000-body disk (seed 1002) that holds a
        bound pair: the group recursion (k_recursion) dominates, ~34,000 sub-steps per step
    python -m paper_2304_07325_gb300.profile_cases steps --n 10000 --steps 4
        the disk stepped one call per step, with each step's recursion sub-steps split by path
        (single-pair / general) -- beside an ncu count of FP64 instructions per k_recursion
        launch, the FP64 instructions per sub-step of each path follow by least squares

Each case prints the per-phase device times measured with CUDA events (symba_profile_step).
"""
from __future__ import annotations

import argparse

from . import PHASES, SYMBA_PRECISION_FP64, SYMBA_PRECISION_MIXED, System, default_params, disk

BOUND_PAIR_GROUP = [1244, 3406, 4643, 5122, 9870]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["step", "bound_pair", "steps"])
    ap.add_argument("--n", type=int, default=10000)
    ap.add_argument("--seed", type=int, default=1002)
    ap.add_argument("--n-field", type=int, default=0, help="step / steps: massless field particles")
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    a = ap.parse_args(argv)
    prec = SYMBA_PRECISION_MIXED if a.precision == "mixed" else SYMBA_PRECISION_FP64
    d = disk.planetesimal_disk(10000 if a.case == "bound_pair" else a.n, a.seed,
                               n_field=0 if a.case == "bound_pair" else a.n_field)
    if a.case == "bound_pair":
        g = BOUND_PAIR_GROUP
        s = System(d.x[g], d.v[g], d.m[g], d.radius[g], params=default_params(precision=prec))
    else:
        s = System(d.x, d.v, d.m, d.radius, n_massive=d.n_massive, params=default_params(precision=prec))
    if a.case == "steps":
        print("step substeps pair_substeps general_substeps max_chain recursion_ms")
        status = 0
        for k in range(a.steps):
            ph = s.profile_step(1)
            st = s.stats()
            status = s.sync()
            print(f"{k} {st.substeps} {st.pair_substeps} {st.substeps - st.pair_substeps} {st.max_chain} {ph[5]:.3f}")
        s.close()
        return 0 if status >= 0 else 1
    ph = s.profile_step(a.steps)
    st = s.stats()
    status = s.sync()
    print(f"case {a.case} status {status} substeps {st.substeps} depth {st.max_depth} "
          f"longest chain {st.max_chain} single-pair path {st.pair_substeps}")
    for name, ms in zip(PHASES, ph):
        print(f"  {name:28s} {ms:10.3f} ms")
    if st.substeps:
        print(f"  recursion per sub-step      {1e3 * ph[5] / st.substeps:10.3f} us")
        print(f"  per longest-chain sub-step  {1e3 * ph[5] / st.max_chain:10.3f} us")
    s.close()
    return 0 if status >= 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
