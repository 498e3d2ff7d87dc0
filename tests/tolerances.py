"""Parity gates shared by the GPU tests (normwise per function:
max |gpu - oracle| / max |oracle| over one function's outputs).

FP64    1e-12  the FP64 target; the same sums taken in another order differ
               by ~1e-15 * sqrt(terms) (measured <= 3e-15 at B = 128).
FP32    2e-5   FP32 unit round-off 6e-8 times the ~sqrt(2B) log2(2B) growth of
               three chained sums of up to 2B terms, with margin.
SPLIT   1e-6   the bound stated for the split-precision tensor-core path
               (TF32x3 and FP16x3: hi/lo pairs of 11 + 11 significant bits,
               three products, FP32 accumulation and FP32 FFT).  A 22-bit
               product pair drops terms of order 2^-22 = 2.4e-7 of each
               product; with FP32 storage of the stage outputs and the FFT's
               round-off the measured round trip at B = 128 x 64 is 6e-7.
               The gate is the target itself, so any regression past it fails.
"""
FP64_TOL = 1e-12
FP32_TOL = 2e-5
SPLIT_TOL = 1e-6
