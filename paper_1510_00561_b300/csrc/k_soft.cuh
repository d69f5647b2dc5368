// k_soft.cuh -- per-subband soft thresholding of a transform plan's
// coefficients (forward and backward), for gradient-based tuning of the
// subband thresholds.
#pragma once
#include <algorithm>
#include <vector>

#include "cvc_internal.cuh"

namespace cvc {

// one block's chunk of coefficients: elements [off, off + n) of the plan's
// coefficient buffer, all in one subband; t = threshold index (-1: lowpass)
struct SoftJob {
    long long off;
    int n;
    int t;
    int pad;
};

constexpr int SOFT_CHUNK = 4096;   // elements per block
constexpr int SOFT_THREADS = 256;

// jobs of a batch of coefficient vectors of layout `lay`; first[s] .. first[s+1]
// are the jobs of directional subband s (first has nsub + 1 entries)
void soft_jobs(const PlaneLayout& lay, int batch, std::vector<SoftJob>* jobs, std::vector<int>* first);

cudaError_t launch_soft_fwd(const SoftJob* d_jobs, int njobs, const float* c, const float* T, float* y,
                            cudaStream_t st);
cudaError_t launch_soft_bwd(const SoftJob* d_jobs, int njobs, const int* d_first, int nsub, const float* c,
                            const float* T, const float* g, float* gc, float* gT, float* d_partial,
                            cudaStream_t st);

}  // namespace cvc
