"""The mixed-precision kick's relative displacement, stated against the FP64-formed-then-rounded
value (CPU only).

The FP32 pair kick does not subtract FP64 positions (three FP64-pipe instructions per pair would
make it FP64-bound); it keeps each position as an FP32 pair x = xf + xl (xf = RN32(x),
xl = RN32(x - xf)) and forms d = (xf_j - xf_i) + (xl_j - xl_i) in FP32.  This test evaluates that
expression with IEEE FP32 arithmetic (numpy float32 rounds every operation to nearest) on the
trapezoid pairs (i massive) of the N = 10,000 benchmark disk and the field-dominated disk and states
its error against RN32(x_j - x_i), the FP64 difference rounded once to FP32:

  - for every pair the level-0 kick weights above zero -- separations beyond the inner shell
    R_1 = lambda (rH_i + rH_j) / 2.08, at least 1.5e-2 AU on these disks (the changeover weight
    g_0 vanishes inside R_1) -- RN32(x_j - x_i) itself or one of its two neighbouring floats
    (at most one FP32 ulp), hence at most 1.5 ulp from the FP64 difference;
  - closer than that, the split's own representation error (2^-48 |x| per position) dominates:
    |d - (x_j - x_i)| <= 2^-47 max(|x_i|, |x_j|) + one ulp of d, several ulps for pairs ~1e-7 AU
    apart, all of them pairs whose level-0 force is weighted by zero.

The source checks at the end tie the expression here to the kernels'."""
import math
import os

import numpy as np

from paper_2304_07325_gb300 import disk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_07325_gb300", "csrc")
LAMBDA, RATIO = 6.5, 2.08


def _hill(d):
    """a (m / 3)^{1/3} from vis-viva with mu = G (1 + m) (heliocentric input state)."""
    G = 4.0 * math.pi ** 2
    r = np.linalg.norm(d.x, axis=1)
    v2 = np.sum(d.v * d.v, axis=1)
    inv_a = 2.0 / r - v2 / (G * (1.0 + d.m))
    a = np.where(inv_a > 0, 1.0 / inv_a, r)
    return a * np.cbrt(d.m / 3.0)


def _pairs(d, rng):
    nm, n = d.n_massive, d.n
    i = rng.integers(0, nm, 600_000)
    j = rng.integers(0, n, 600_000)
    # plus neighbours along x: the closest pairs, where the high parts cancel
    order = np.argsort(d.x[:, 0])
    i = np.concatenate([i, order[:-1]])
    j = np.concatenate([j, order[1:]])
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    keep = (lo != hi) & (lo < nm)              # trapezoid pairs: the lower index is massive
    return lo[keep], hi[keep]


def test_split_displacement_against_fp64_then_rounded():
    rng = np.random.default_rng(7)
    lines = []
    for d in (disk.planetesimal_disk(10000, 1002), disk.planetesimal_disk(1000, 1003, n_field=100000)):
        i, j = _pairs(d, rng)
        x = d.x
        xf = x.astype(np.float32)
        xl = (x - xf.astype(np.float64)).astype(np.float32)
        dd = ((xf[j] - xf[i]) + (xl[j] - xl[i])).astype(np.float64)   # FP32 operations, as in the kernel
        exact = x[j] - x[i]                                             # the FP64 difference
        ref = exact.astype(np.float32).astype(np.float64)               # ... rounded once to FP32
        ulp = np.spacing(np.abs(ref.astype(np.float32))).astype(np.float64)
        rh = _hill(d)
        R1 = LAMBDA * (rh[i] + rh[j]) / RATIO
        assert R1.min() > 1.5e-2
        sep = np.linalg.norm(exact, axis=1)
        far = sep >= R1                                                  # weighted above zero
        e_ref = np.abs(dd - ref) / ulp
        # within one ulp of RN32(x_j - x_i): d is that float or one of its two neighbours
        r32 = ref.astype(np.float32)
        up, down = np.nextafter(r32, np.float32(np.inf)), np.nextafter(r32, np.float32(-np.inf))
        d32 = dd.astype(np.float32)
        assert np.all(((d32 == r32) | (d32 == up) | (d32 == down))[far])
        # against the FP64 difference itself: the half ulp of the reference's rounding plus one ulp
        e_fp64 = np.abs(dd - exact) / ulp
        assert e_fp64[far].max() <= 1.5, e_fp64[far].max()
        near = ~far
        bound = 2.0 ** -47 * np.maximum(np.abs(x[i]), np.abs(x[j])) + np.spacing(np.abs(dd.astype(np.float32))).astype(np.float64)
        assert np.all(np.abs(dd - exact)[near] <= bound[near])
        lines.append(f"{d.label}: {far.sum()} pairs beyond R_1: identical to RN32(FP64 difference) for "
                     f"{100 * np.mean(e_ref[far] == 0):.1f} %, otherwise a neighbouring float; worst "
                     f"{e_fp64[far].max():.2f} ulp from the FP64 difference; {near.sum()} closer pairs (weight 0): worst "
                     f"{e_ref[near].max() if near.any() else 0:.2f} ulp")
        assert np.mean(e_ref[far] == 0) > 0.5
    print("\n".join(lines))


def test_the_kernels_use_this_expression():
    trap = open(os.path.join(CSRC, "k_trap.cu")).read()
    misc = open(os.path.join(CSRC, "k_misc.cu")).read()
    for c in "xyz":
        # the trapezoid tiles (row r, column j) and the field rectangle (source q, field particle p)
        assert f"const float d{c} = ({c}hj - r.{c}h) + ({c}lj - r.{c}l);" in trap
        assert f"const float d{c} = (q.{c}f - {c}hp) + (q.{c}l - {c}lp);" in trap
        assert f"D.{c}l[p] = __double2float_rn({c} - (double)f{c});" in misc
