// k_lift.cu -- lifting passes of the directional filter bank (§2.1).
//
// Every DFB stage is a two-channel fan filter bank in ladder form: a
// predict pass on one coset of the channel's samples and an update pass on
// the other, each a 16-tap stencil of the other coset.  The host builds one
// job per target coset array (with the stencil already mapped to that
// array's coordinates), and one launch runs one pass of one stage for every
// plane, pyramid level and channel at once.  One thread computes one
// target sample:
//   out(u,v) = alpha * tin(u,v) + gamma * sum_t w[t] * src_sel[t](u+dr[t], v+dc[t])   (periodic)
#include "cvc_internal.cuh"

namespace cvc {

__device__ __forceinline__ int wrap_l(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    int r = a % n;
    return r < 0 ? r + n : r;
}

constexpr int LIFT_BLOCK = 256;

__global__ void __launch_bounds__(LIFT_BLOCK) k_lift(const LiftJob* __restrict__ jobs,
                                                     const int* __restrict__ block_job, Bases B) {
    __shared__ LiftJob J;
    const int jid = block_job[blockIdx.x];
    {
        const int* src = reinterpret_cast<const int*>(jobs + jid);
        int* dst = reinterpret_cast<int*>(&J);
        for (int i = threadIdx.x; i < (int)(sizeof(LiftJob) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const long long e = (long long)(blockIdx.x - J.first_block) * LIFT_BLOCK + threadIdx.x;
    const int rows = J.rows, cols = J.cols;
    if (e >= (long long)rows * cols) return;
    const int u = (int)(e / cols), v = (int)(e - (long long)u * cols);
    const float* s0 = B.p[J.src[0].b] + J.src[0].off;
    const float* s1 = B.p[J.src[1].b] + J.src[1].off;
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 16; t++) {
        const int r = wrap_l(u + J.dr[t], rows), c = wrap_l(v + J.dc[t], cols);
        const float* s = J.sel[t] ? s1 : s0;
        const int rs = J.sel[t] ? J.src[1].rs : J.src[0].rs;
        const int cs = J.sel[t] ? J.src[1].cs : J.src[0].cs;
        acc = fmaf(J.w[t], s[(long long)r * rs + (long long)c * cs], acc);
    }
    const float tv = B.p[J.tin.b][J.tin.off + (long long)u * J.tin.rs + (long long)v * J.tin.cs];
    B.p[J.out.b][J.out.off + (long long)u * J.out.rs + (long long)v * J.out.cs] = fmaf(J.alpha, tv, J.gamma * acc);
}

cudaError_t launch_lift(const LaunchLift& L, Bases bases, cudaStream_t st) {
    if (L.nblocks == 0) return cudaSuccess;
    k_lift<<<L.nblocks, LIFT_BLOCK, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    return cudaGetLastError();
}

}  // namespace cvc
