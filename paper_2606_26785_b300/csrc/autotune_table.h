// Tuned choices of the mixed-precision inverse-Lanczos path per matrix order,
// written by paper_2606_26785_b300/probe/tune.py (an offline sweep over the FP32
// solver kernel and the number of Lanczos slots on one GPU).  Entry i applies
// to n <= n_max[i] (the last entry to every larger n).
// sweep: NVIDIA B300 SXM6 AC, 2026-12-04; 64 x 64 grid, mixed precision, rtol 1e-8
#pragma once
namespace pseudo {
struct TunePoint {
    int n_max;        // largest matrix order of the bucket
    int fp32_solver;  // 0 tensor cores (tcgen05), 1 CUDA cores
    int slots;        // Lanczos slots (shifts per solve launch)
};
static const TunePoint kTuneTable[] = {
    {304, 0, 8192},  // n = 256: 450018 points/s
    {431, 0, 8192},  // n = 362: 300688 points/s
    {609, 0, 8192},  // n = 512: 215982 points/s
    {861, 0, 8192},  // n = 724: 119090 points/s
    {1218, 0, 8192},  // n = 1024: 100464 points/s
    {1722, 0, 8192},  // n = 1448: 52594 points/s
    {2888, 0, 8192},  // n = 2048: 27176 points/s
    {1 << 30, 0, 8192},  // larger orders: not swept (the defaults)
};
}  // namespace pseudo
