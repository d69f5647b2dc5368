// k_soft.cu -- soft thresholding of contourlet coefficients with one
// threshold per directional subband, and its backward pass.
//
//   forward:  y = sign(c) * max(|c| - T_s, 0) in directional subband s; the
//             lowpass passes through unchanged
//   backward: dL/dc = g * [|c| > T_s] (lowpass: g);
//             dL/dT_s = -sum over subband s (all batch entries) of g * sign(c) * [|c| > T_s]
//
// The threshold gradient is reduced deterministically: every block writes
// the fixed-order sum of its chunk, and one block per subband adds the
// partial sums of that subband's chunks in double precision, in order.
#include "k_soft.cuh"

namespace cvc {

namespace {

__device__ __forceinline__ float soft(float v, float th) { return copysignf(fmaxf(fabsf(v) - th, 0.0f), v); }

__global__ void k_soft_fwd(const SoftJob* __restrict__ jobs, const float* c, const float* __restrict__ T,
                           float* y) {
    const SoftJob J = jobs[blockIdx.x];
    const float* src = c + J.off;
    float* dst = y + J.off;
    if (J.t < 0) {
        for (int i = threadIdx.x; i < J.n; i += blockDim.x) dst[i] = src[i];
        return;
    }
    const float th = T[J.t];
    for (int i = threadIdx.x; i < J.n; i += blockDim.x) dst[i] = soft(src[i], th);
}

__global__ void k_soft_bwd(const SoftJob* __restrict__ jobs, const float* __restrict__ c,
                           const float* __restrict__ T, const float* g, float* gc, float* __restrict__ partial) {
    __shared__ float wsum[SOFT_THREADS / 32];
    const SoftJob J = jobs[blockIdx.x];
    const float* cs = c + J.off;
    const float* gs = g + J.off;
    float* out = gc + J.off;
    if (J.t < 0) {
        for (int i = threadIdx.x; i < J.n; i += blockDim.x) out[i] = gs[i];
        if (threadIdx.x == 0) partial[blockIdx.x] = 0.0f;
        return;
    }
    const float th = T[J.t];
    float acc = 0.0f;
    for (int i = threadIdx.x; i < J.n; i += blockDim.x) {
        const float v = cs[i], gi = gs[i];
        const bool on = fabsf(v) > th;
        out[i] = on ? gi : 0.0f;
        if (on) acc -= (v > 0.0f) ? gi : ((v < 0.0f) ? -gi : 0.0f);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < SOFT_THREADS / 32; w++) s += wsum[w];
        partial[blockIdx.x] = s;
    }
}

// one block per directional subband: its chunks' partial sums, in order
__global__ void k_soft_reduce(const int* __restrict__ first, const float* __restrict__ partial,
                              float* __restrict__ gT) {
    __shared__ double sh[SOFT_THREADS];
    const int s = blockIdx.x;
    const int b0 = first[s], b1 = first[s + 1];
    double acc = 0.0;
    for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) acc += (double)partial[b];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = SOFT_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gT[s] = (float)sh[0];
}

}  // namespace

void soft_jobs(const PlaneLayout& lay, int batch, std::vector<SoftJob>* jobs, std::vector<int>* first) {
    jobs->clear();
    first->clear();
    // lowpass chunks first (pass-through), then subband by subband over the batch
    const SubbandG& low = lay.sb[0];
    for (int b = 0; b < batch; b++) {
        const long long base = (long long)b * lay.total + low.off, n = (long long)low.h * low.w;
        for (long long o = 0; o < n; o += SOFT_CHUNK)
            jobs->push_back({base + o, (int)std::min<long long>(SOFT_CHUNK, n - o), -1, 0});
    }
    for (size_t s = 1; s < lay.sb.size(); s++) {
        first->push_back((int)jobs->size());
        const SubbandG& sb = lay.sb[s];
        for (int b = 0; b < batch; b++) {
            const long long base = (long long)b * lay.total + sb.off, n = (long long)sb.h * sb.w;
            for (long long o = 0; o < n; o += SOFT_CHUNK)
                jobs->push_back({base + o, (int)std::min<long long>(SOFT_CHUNK, n - o), (int)s - 1, 0});
        }
    }
    first->push_back((int)jobs->size());
}

cudaError_t launch_soft_fwd(const SoftJob* d_jobs, int njobs, const float* c, const float* T, float* y,
                            cudaStream_t st) {
    if (njobs == 0) return cudaSuccess;
    k_soft_fwd<<<njobs, SOFT_THREADS, 0, st>>>(d_jobs, c, T, y);
    return cudaGetLastError();
}

cudaError_t launch_soft_bwd(const SoftJob* d_jobs, int njobs, const int* d_first, int nsub, const float* c,
                            const float* T, const float* g, float* gc, float* gT, float* d_partial,
                            cudaStream_t st) {
    if (njobs == 0) return cudaSuccess;
    k_soft_bwd<<<njobs, SOFT_THREADS, 0, st>>>(d_jobs, c, T, g, gc, d_partial);
    if (nsub > 0) k_soft_reduce<<<nsub, SOFT_THREADS, 0, st>>>(d_first, d_partial, gT);
    return cudaGetLastError();
}

}  // namespace cvc
