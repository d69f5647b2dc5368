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
// Passes of the synthesis direction (inverse and adjoint of the forward)
// accumulate the 16 products in float-float (error-free TwoSum / TwoProd):
// their O-coset update doubles the incoming values at every stage, so plain
// single-precision sums would grow the reconstruction error with the tree
// depth.  alpha and gamma are powers of two, so only the final store rounds.
#include "cvc_internal.cuh"

namespace cvc {

__device__ __forceinline__ int wrap_l(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    int r = a % n;
    return r < 0 ? r + n : r;
}

constexpr int LIFT_BLOCK = 256;

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    float s = __fadd_rn(hi, x);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

template <bool COMP>
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
    float acc = 0.f, lo = 0.f;
#pragma unroll
    for (int t = 0; t < 16; t++) {
        const int r = wrap_l(u + J.dr[t], rows), c = wrap_l(v + J.dc[t], cols);
        const float* s = J.sel[t] ? s1 : s0;
        const int rs = J.sel[t] ? J.src[1].rs : J.src[0].rs;
        const int cs = J.sel[t] ? J.src[1].cs : J.src[0].cs;
        const float x = s[(long long)r * rs + (long long)c * cs];
        if (COMP) {
            const float p = __fmul_rn(J.w[t], x);
            const float pe = fmaf(J.w[t], x, -p);
            two_sum_acc(acc, lo, p);
            lo = __fadd_rn(lo, pe);
        } else {
            acc = fmaf(J.w[t], x, acc);
        }
    }
    const float tv = B.p[J.tin.b][J.tin.off + (long long)u * J.tin.rs + (long long)v * J.tin.cs];
    float res;
    if (COMP) {
        float hi = __fmul_rn(J.gamma, acc), l2 = __fmul_rn(J.gamma, lo);  // exact: gamma is a power of two
        two_sum_acc(hi, l2, __fmul_rn(J.alpha, tv));                      // exact: alpha is a power of two
        res = __fadd_rn(hi, l2);
    } else {
        res = fmaf(J.alpha, tv, J.gamma * acc);
    }
    B.p[J.out.b][J.out.off + (long long)u * J.out.rs + (long long)v * J.out.cs] = res;
}

cudaError_t launch_lift(const LaunchLift& L, Mode m, Bases bases, cudaStream_t st) {
    if (L.nblocks == 0) return cudaSuccess;
    if (m == INV || m == FWD_ADJ) k_lift<true><<<L.nblocks, LIFT_BLOCK, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    else k_lift<false><<<L.nblocks, LIFT_BLOCK, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    return cudaGetLastError();
}

}  // namespace cvc
