// Tuned choices of the mixed-precision inverse-Lanczos path per matrix order,
// written by paper_2606_26785_b300/probe/tune.py (an offline sweep over the FP32
// solver kernel and the number of Lanczos slots on one GPU).  Entry i applies
// to n <= n_max[i] (the last entry to every larger n).
// sweep: not run yet (the entries below are the untuned defaults)
#pragma once
namespace pseudo {
struct TunePoint {
    int n_max;        // largest matrix order of the bucket
    int fp32_solver;  // 0 tensor cores (tcgen05), 1 CUDA cores
    int slots;        // Lanczos slots (shifts per solve launch)
};
static const TunePoint kTuneTable[] = {
    {1 << 30, 0, 8192},
};
}  // namespace pseudo
