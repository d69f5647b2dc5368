// k_tail.cu -- the pyramid tail: a plane's coarse levels in one block (§2.1,
// Fig. 1: the LP iterated on the lowpass, a DFB on every detail image).
//
// Where a plane's levels t..L fit in one block's shared memory (their detail
// images, DFB partner buffers and lowpass images), a single block runs all
// of their steps: in the forward direction the LP analysis of level t (its
// input lowpass read from global memory), the DFB stages of its detail, the
// LP analysis of level t+1 on the resident lowpass, and so on to level L,
// writing only coefficients; in the inverse direction the DFB synthesis and
// LP synthesis of levels L..t, writing only level t's output lowpass (as a
// (hi, lo) pair) for the next launch.  Every step is the same tile
// computation as the per-level launches (lp_tile.cuh, dfb_tile.cuh), so a
// plane gives the same bits whichever levels its tail takes; what changes
// is that the intermediate images stay on chip and that the coarse levels,
// whose per-level launches would each be a few blocks, take one launch.
#include <mutex>

#include "dfb_tile.cuh"
#include "lp_tile.cuh"

namespace cvc {

namespace {

constexpr int kMaxDynSmem = 232448;   // bytes of shared memory a block may use (sm_100 family)

// tile scratch of every step kind, in floats, each array 16-byte aligned
template <int NT>
constexpr int b_array_floats() { return (BGeo<NT>::SMB + 3) & ~3; }
template <int NT>
constexpr int scratch_floats() {
    static_assert(LevelGeo<4, 3>::FLOATS <= (int)(ff_smem<4, 3>() / 4), "the single-precision tile fits the scratch");
    constexpr int lp = (int)(ff_smem<4, 3>() / 4);
    constexpr int a = AGeo<NT>::SMEM / 4;
    constexpr int b = 2 * b_array_floats<NT>();
    return (((lp > a ? lp : a) > b ? (lp > a ? lp : a) : b) + 3) & ~3;
}

__device__ __forceinline__ int lp_tiles(const LpJob& J) { return ((J.H + LP_TILE - 1) / LP_TILE) * J.tiles_x; }
__device__ __forceinline__ int a_tiles(const DfbAJob& J) { return ((J.H + DFBA_TILE - 1) / DFBA_TILE) * J.tiles_x; }
__device__ __forceinline__ int b_tiles(const DfbBJob& J) { return ((J.R2 + DFBB_ROWS - 1) / DFBB_ROWS) * J.tiles_x; }

// one block per plane; dynamic shared memory: the tile scratch, then the plane's resident workspace
template <bool SYN, int NT>
__global__ void __launch_bounds__(256, 1) k_pyr_tail(const TailPlane* __restrict__ planes,
                                                  const TailStep* __restrict__ steps, const LpJob* __restrict__ lp,
                                                  const DfbAJob* __restrict__ da, const DfbBJob* __restrict__ db,
                                                  Bases B, PassParams pp) {
    extern __shared__ __align__(16) float sm[];
    const TailPlane& T = planes[blockIdx.x];
    if (job_idle(B, T.stream)) return;
    Bases Bt = B;
    Bt.p[B_SMEM] = sm + scratch_floats<NT>();
    constexpr int BA = b_array_floats<NT>();
    for (int s = 0; s < T.nsteps; s++) {
        const TailStep st = steps[T.first_step + s];
        if (st.kind == 0) {
            const LpJob& J = lp[st.job];
            const int n = lp_tiles(J);
            for (int tile = 0; tile < n; tile++) {
                __syncthreads();   // the previous tile is done with the scratch
                if (st.centred) {
                    // the first level: centred single precision, as its own launches run it
                    using LG = LevelGeo<4, 3>;
                    float* s_a = sm + ((LG::MN * LG::MNS + 3) & ~3);
                    lp_level_tile<4, 3, true, SYN>(J, tile, Bt, sm, s_a, s_a + ((LG::NA + 3) & ~3));
                } else {
                    lp_ff_tile<4, 3, !SYN>(J, tile, Bt, sm);
                }
            }
        } else if (st.kind == 1) {
            const DfbAJob& J = da[st.job];
            const int n = a_tiles(J);
            for (int tile = 0; tile < n; tile++) {
                __syncthreads();
                dfb_a_tile<SYN, NT>(J, tile, Bt, pp, sm);
            }
        } else {
            const DfbBJob& J = db[st.job];
            const int n = b_tiles(J);
            for (int tile = 0; tile < n; tile++) {
                __syncthreads();
                if (pp.first_odd) dfb_b_tile<SYN, NT, true, true, 256>(J, tile, Bt, pp, sm, sm + BA);
                else dfb_b_tile<SYN, NT, false, true, 256>(J, tile, Bt, pp, sm, sm + BA);
            }
        }
        __syncthreads();   // the step's resident outputs are complete before the next step reads them
    }
}

template <bool SYN, int NT>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_pyr_tail<SYN, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

}  // namespace

int tail_ws_budget(int ntaps) {
    const int scratch = ntaps == 8 ? scratch_floats<8>() : ntaps == 6 ? scratch_floats<6>() : scratch_floats<4>();
    return kMaxDynSmem / 4 - scratch;
}

cudaError_t tail_prepare() {
    static std::once_flag once;
    static cudaError_t status = cudaSuccess;
    std::call_once(once, [] {
        status = set_attr<false, 4>();
        if (status == cudaSuccess) status = set_attr<true, 4>();
        if (status == cudaSuccess) status = set_attr<false, 6>();
        if (status == cudaSuccess) status = set_attr<true, 6>();
        if (status == cudaSuccess) status = set_attr<false, 8>();
        if (status == cudaSuccess) status = set_attr<true, 8>();
    });
    return status;
}

cudaError_t launch_tail(const LaunchTail& L, Mode m, Bases bases, cudaStream_t st) {
    if (L.nplanes == 0) return cudaSuccess;
    if (m != FWD && m != INV) return cudaErrorInvalidValue;
    cudaError_t e = tail_prepare();
    if (e != cudaSuccess) return e;
    const bool syn = m == INV;
    const PassParams pp = pass_params(m);
    const int nt = L.ntaps;
    const int scratch = nt == 8 ? scratch_floats<8>() : nt == 6 ? scratch_floats<6>() : scratch_floats<4>();
    const size_t smem = sizeof(float) * (size_t)(scratch + L.ws_floats);
    if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
#define CVC_TAIL(S, N) \
    k_pyr_tail<S, N><<<L.nplanes, 256, smem, st>>>(L.d_planes, L.d_steps, L.d_lp, L.d_a, L.d_b, bases, pp)
    if (nt == 6) {
        if (syn) CVC_TAIL(true, 6);
        else CVC_TAIL(false, 6);
    } else if (nt == 8) {
        if (syn) CVC_TAIL(true, 8);
        else CVC_TAIL(false, 8);
    } else {
        if (syn) CVC_TAIL(true, 4);
        else CVC_TAIL(false, 4);
    }
#undef CVC_TAIL
    return cudaGetLastError();
}

}  // namespace cvc
