// Tuned choices of the mixed-precision inverse-Lanczos path per matrix order,
// written by paper_2606_26785_b300/probe/tune.py (an offline sweep over the FP32
// solver kernel, with the tensor-core solve's column-group form, and the number
// of Lanczos slots on one GPU).  Entry i applies to n <= n_max[i] (the last
// entry to every larger n).
// sweep: NVIDIA B300 SXM6 AC, 2026-12-04; 64 x 64 grid, mixed precision, rtol 1e-8.
// That sweep chose the tensor cores (over the CUDA cores) and 8192 slots in every
// bucket; the tensor-core form of these buckets (16 right-hand sides per CTA, 3)
// comes from the solve sweep of both forms on the same part (probe/solve_sweep.py:
// the 16-column form 1.2-1.6x faster than the 32-column one at orders 256 .. 2048),
// and larger orders keep the form by order (0: 32 columns from padded order 4096,
// 1.12x and 1.16-1.31x faster at n = 4000 and 8000).
#pragma once
namespace pseudo {
struct TunePoint {
    int n_max;        // largest matrix order of the bucket
    int fp32_solver;  // 0 tensor cores (form by order), 1 CUDA cores, 3 / 4 tensor cores,
                      // 16 / 32 right-hand sides per CTA
    int slots;        // Lanczos slots (shifts per solve launch)
};
static const TunePoint kTuneTable[] = {
    {304, 3, 8192},  // n = 256: 450018 points/s
    {431, 3, 8192},  // n = 362: 300688 points/s
    {609, 3, 8192},  // n = 512: 215982 points/s
    {861, 3, 8192},  // n = 724: 119090 points/s
    {1218, 3, 8192},  // n = 1024: 100464 points/s
    {1722, 3, 8192},  // n = 1448: 52594 points/s
    {2888, 3, 8192},  // n = 2048: 27176 points/s
    {1 << 30, 0, 8192},  // larger orders: not swept (the defaults)
};
}  // namespace pseudo
