"""One pass of a named workload at a profiler-friendly size (for ncu captures).

    python -m paper_1507_00895_gb300.profile_case <case>

Cases (inputs from paper_1507_00895_gb300.inputs; every stage runs in libdf):
  mixed64  2D 16x16, n_w = 64, N_W = 15, DF_FP32_IR: bubble + both ladder
           channels (7,680 ladders of order 64, bse_mixed_kernel)
  bench64  the benchmark's workload itself (2D 32x32, n_w = 64, N_W = 15),
           DF_FP32_IR: bubble + both ladder channels (30,720 ladders)
  tc96     3D 8^3, n_w = 96, N_W = 5, DF_FP32_IR: bubble + both ladder channels
           (5,120 ladders of order 96, the tensor-core Gauss-Jordan kernel)
  simt96   the same with the CUDA-core Gauss-Jordan (mixed_sweep = 1)
  fft3d    3D 16^3, n_w = 96, N_W = 21 (the 3D workload at its stated size), FP64:
           Eq. dual_bubble and Eq. sd + Dyson only (the lattice-FFT kernels;
           ladders skipped, the kernel array stays zero)
Each case runs its stages once after one untimed warm-up pass, then prints the
device time of each stage group (libdf's CUDA events).
"""
from __future__ import annotations

import sys


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    case = argv[0] if argv else "tc96"
    from paper_1507_00895_gb300 import build, df, inputs as I
    build.build_lib()
    if case == "mixed64":
        w, kw, stages = I.workload("square32_tp", nk=16), dict(precision=df.DF_FP32_IR), ("bubble", "bse")
    elif case == "bench64":
        w, kw, stages = I.workload("square32_tp"), dict(precision=df.DF_FP32_IR), ("bubble", "bse")
    elif case in ("tc96", "simt96"):
        w = I.workload("cubic16_crit", nk=8, m_max=2)
        kw = dict(precision=df.DF_FP32_IR, mixed_sweep=0 if case == "tc96" else 1)
        stages = ("bubble", "bse")
    elif case == "fft3d":
        w, kw, stages = I.workload("cubic16_crit"), dict(eig_mode=0), ("bubble", "sigma")
    else:
        print(f"unknown case {case!r}", file=sys.stderr)
        return 2
    with df.DualFermion.from_workload(w, **kw) as d:
        for rep in range(2):
            if rep == 1:
                d.set_timing(True)
            for s in stages:
                if s == "bubble":
                    d.bubble()
                elif s == "bse":
                    d.bse(3)
                else:
                    d.sigma(want_residual=False)
        t = d.get_timing()
    print(case, {k: round(v[0], 4) for k, v in t.items() if v[1]})
    return 0


if __name__ == "__main__":
    sys.exit(main())
