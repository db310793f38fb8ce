"""Writes fcsph_roots.cuh: cos(2 pi e / N) and sin(2 pi e / N), e < N, as
switch tables for the composite sizes of the register column FFT
(fcsph_regfft.cuh).  The values are computed in 40-digit arithmetic (mpmath)
and printed with 17 significant digits; with a compile-time e the switch folds
to an immediate.  Run from this directory after changing SIZES:

    python gen_roots.py
"""
import os

import mpmath as mp

SIZES = [6, 10, 14, 15, 20, 21, 25, 27, 28, 30, 35, 36, 42, 50]


def main():
    mp.mp.dps = 40
    out = ["// Generated by gen_roots.py: cos and sin of 2 pi e / N for the composite",
           "// register-DFT sizes N.  Do not edit by hand.",
           "#pragma once", "", "namespace fcsph {", "",
           "template <int N> __device__ __forceinline__ float rcos(int e);",
           "template <int N> __device__ __forceinline__ float rsin(int e);", ""]
    for n in SIZES:
        for name, fn in (("rcos", mp.cos), ("rsin", mp.sin)):
            out.append(f"template <> __device__ __forceinline__ float {name}<{n}>(int e) {{")
            out.append(f"  switch (((e % {n}) + {n}) % {n}) {{")
            for e in range(n):
                v = fn(2 * mp.pi * e / n)
                out.append(f"    case {e}: return {mp.nstr(v, 17, min_fixed=-2, max_fixed=2)}f;")
            out.append("    default: return 0.0f;")
            out.append("  }")
            out.append("}")
        out.append("")
    out.append("}  // namespace fcsph")
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "fcsph_roots.cuh"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
