// static_lp.cu -- an allocation-free entry point: the Laplacian-pyramid
// forward transform with its scratch in a fixed device array.
//
// Who needs it: callers that cannot allocate device memory while they run --
// e.g. code that owns a fixed memory budget handed out up front, or runs
// where the CUDA allocator is off limits -- cannot create a cvc_ct_plan
// (which cudaMallocs its workspace and job tables).  This entry point makes
// no allocation of any kind: the intermediate lowpass images, the per-level
// job records and the tile-to-job map live in one file-scope __device__
// array that every GPU loading the library holds until the process exits.
#include <atomic>
#include <cstring>

#include "cvc_internal.cuh"

using namespace cvc;

namespace {

// size of the shared scratch array: 4 Mi floats (16 MiB) in all
constexpr long long kStaticFloats = 4LL << 20;
// layout: [job records: one per level][tile-to-job map][lowpass workspace]
constexpr int kJobSlotFloats = 64;  // >= sizeof(LpJob) / 4, 256-byte slots
constexpr int kMaxTiles = 16384;    // level-1 tiles of 64 x 64 (e.g. 8192 x 8192)
constexpr long long kWorkOffset = CVC_MAX_LEVELS * kJobSlotFloats + kMaxTiles;
constexpr long long kWorkFloats = kStaticFloats - kWorkOffset;
static_assert(sizeof(LpJob) <= kJobSlotFloats * 4, "job slot too small");

static __device__ __align__(256) float g_lp_scratch[kStaticFloats];

// the device address of g_lp_scratch, looked up once per device
constexpr int kMaxDevices = 64;
std::atomic<float*> g_scratch_ptr[kMaxDevices];

// every level's job record, passed by value to the set-up kernel
struct StaticJobs {
    LpJob job[CVC_MAX_LEVELS];
    int levels;
};

// writes the job records into their slots and zeroes the tile-to-job map
// (every tile of a launch belongs to that launch's single job)
__global__ void k_static_setup(StaticJobs jobs, float* base, int tiles) {
    int* block_job = reinterpret_cast<int*>(base + CVC_MAX_LEVELS * kJobSlotFloats);
    for (int i = threadIdx.x; i < tiles; i += blockDim.x) block_job[i] = 0;
    if (threadIdx.x < jobs.levels)
        *reinterpret_cast<LpJob*>(base + threadIdx.x * kJobSlotFloats) = jobs.job[threadIdx.x];
}

}  // namespace

extern "C" cvc_status cvc_lp_pyramid_forward_static(const float* d_x, int h, int w, int levels, float* d_coeffs,
                                                    cvc_stream_t stream) {
    if (!d_x || !d_coeffs || levels < 1 || levels > CVC_MAX_LEVELS || h <= 0 || w <= 0) return CVC_ERR_INVALID_ARG;
    if (h % (1 << levels) || w % (1 << levels)) return CVC_ERR_INVALID_ARG;
    // limits of the fixed array
    long long need = 0;
    for (int j = 1; j < levels; j++) need += (long long)(h >> j) * (w >> j);
    const long long tiles1 = (long long)((h + LP_TILE - 1) / LP_TILE) * ((w + LP_TILE - 1) / LP_TILE);
    if (need > kWorkFloats || tiles1 > kMaxTiles) return CVC_ERR_UNSUPPORTED;
    // set-up, once per device with that device current: the device address of the array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CVC_ERR_CUDA;
    float* base = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!base) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lp_scratch) != cudaSuccess || !p) return CVC_ERR_CUDA;
        base = static_cast<float*>(p);
        g_scratch_ptr[dev].store(base, std::memory_order_release);   // racing first calls store the same value
    }
    cudaStream_t st = (cudaStream_t)stream;
    Bases B;
    memset(&B, 0, sizeof(B));
    B.p[B_IN] = const_cast<float*>(d_x);
    B.p[B_COEF] = d_coeffs;
    B.p[B_WORK] = base + kWorkOffset;
    // coefficient layout of cvc_ct_layout with dirs_log2 = 0: lowpass, then the detail of each level
    StaticJobs jobs;
    memset(&jobs, 0, sizeof(jobs));
    jobs.levels = levels;
    long long coff = (long long)(h >> levels) * (w >> levels);
    long long woff = 0, prev_woff = 0;
    for (int j = 1; j <= levels; j++) {
        const int hj = h >> (j - 1), wj = w >> (j - 1);
        LpJob& J = jobs.job[j - 1];
        J.H = hj;
        J.W = wj;
        J.tiles_x = (wj + LP_TILE - 1) / LP_TILE;
        J.first_block = 0;
        J.main.b = j == 1 ? B_IN : B_WORK;
        J.main.off = j == 1 ? 0 : prev_woff;
        J.main.rs = wj;
        J.main.cs = 1;
        J.cout.b = j == levels ? B_COEF : B_WORK;
        J.cout.off = j == levels ? 0 : woff;
        J.cout.rs = wj / 2;
        J.cout.cs = 1;
        J.out.b = B_COEF;
        J.out.off = coff;
        J.out.rs = wj;
        J.out.cs = 1;
        J.cin_lo.b = -1;
        J.out_lo.b = -1;
        J.stream = -1;
        coff += (long long)hj * wj;
        prev_woff = woff;
        woff += (long long)(hj / 2) * (wj / 2);
    }
    k_static_setup<<<1, 256, 0, st>>>(jobs, base, (int)tiles1);
    if (cudaGetLastError() != cudaSuccess) return CVC_ERR_CUDA;
    note_launches(1);
    int* block_job = reinterpret_cast<int*>(base + CVC_MAX_LEVELS * kJobSlotFloats);
    for (int j = 1; j <= levels; j++) {
        const int hj = h >> (j - 1);
        LaunchLp L;
        L.njobs = 1;
        L.centred = j == 1;   // as the plan's forward first level
        L.nblocks = ((hj + LP_TILE - 1) / LP_TILE) * jobs.job[j - 1].tiles_x;
        L.d_jobs = reinterpret_cast<LpJob*>(base + (j - 1) * kJobSlotFloats);
        L.d_block_job = block_job;
        if (launch_lp(L, FWD, B, st) != cudaSuccess) return CVC_ERR_CUDA;
        note_launches(1);
    }
    return CVC_OK;
}
