// cvc_internal.cuh -- shared device/host declarations of the CUDA codec path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/cvc.h"

namespace cvc {

// ------------------------------------------------------------ error flags
// Device-detected conditions are OR-ed into a per-context status word.
enum : uint32_t {
    EF_OVERFLOW = 1u << 0,  // quantised code outside int16
    EF_CAPACITY = 1u << 1,  // token stream exceeds the output buffer
    EF_CORRUPT = 1u << 2,   // malformed bitstream
    EF_MISMATCH = 1u << 3,  // bitstream header does not match the codec
    EF_STATE = 1u << 4,     // P-frame without its reference
};

// Base pointers of one transform invocation; job tables address memory as
// (base id, element offset) so that the tables stay valid across calls.
// `act` (may be NULL) marks the streams that take part in the call: stream
// s takes part iff the int at byte offset s * act_stride is non-zero; the
// tile kernels skip the jobs of the other streams (a job's stream < 0: always).
// B_SMEM: inside the pyramid-tail kernel, the block's resident workspace in shared memory.
enum { B_IN = 0, B_COEF = 1, B_WORK = 2, B_OUT = 3, B_SMEM = 4, N_BASES = 5 };
struct Bases {
    float* p[N_BASES];
    const int* act;
    int act_stride;
};

// the job's stream does not take part in this call: the whole block returns
__device__ __forceinline__ bool job_idle(const Bases& B, int stream) {
    return B.act != nullptr && stream >= 0 &&
           *reinterpret_cast<const int*>(reinterpret_cast<const char*>(B.act) + (size_t)stream * B.act_stride) == 0;
}

// Base pointer b, chosen by selects: a run-time index into a by-value kernel
// parameter makes the compiler copy the whole parameter to the stack and
// every thread read it back from local memory.
__device__ __forceinline__ float* base_ptr(const Bases& B, int b) {
    float* p = B.p[0];
#pragma unroll
    for (int k = 1; k < N_BASES; k++) p = b == k ? B.p[k] : p;
    return p;
}

// Strided 2-D view: element (u, v) is at base[b] + off + u*rs + v*cs.
struct View {
    long long off;
    int b;
    int rs, cs;
};

// Directional filter bank jobs.  Each DFB stage is a two-channel fan filter
// bank in ladder form: a pass over one coset of a channel's samples (the
// "target" parity) followed by a pass over the other, each sample becoming
//   alpha * itself + gamma * (16-tap stencil of the other coset).
// The mode fixes which parity goes first and the (alpha, gamma) pairs.
struct PassParams {
    int first_odd;      // 1: the odd coset is the first target
    float a1, g1, a2, g2;
};

// Stages 1 and 2 of one detail image, fused in 64 x 64 tiles.  The stage-2
// channels are the image's polyphase classes q = 2*(row & 1) + (col & 1);
// comp[q] is where class q lives outside the image: the children in the
// analysis direction, the inputs in the synthesis direction.  nst = 1 runs
// stage 1 only (its cosets, classes {00, 11} and {01, 10}, are then the
// subbands and comp[] points into them).
struct DfbAJob {
    View D;        // H x W detail image (rs = pitch, cs = 1)
    View comp[4];  // (H/2) x (W/2) each, any strides
    int H, W;
    int nst;
    int tiles_x, first_block;
    int ntaps;     // prototype length (4, 6 or 8)
    int stream;    // the plane's stream (Bases::act), -1: none
};

// One stage s >= 3 of one channel: its array splits into even / odd rows,
// R2 x C each, under the 4 x 4 stencil of slope index i (row offset a, column
// offset -i*a + (b-a)/2).  Family-r channels are kept transposed so the same
// job serves both families.
struct DfbBJob {
    View pe, po;   // parent's even / odd rows
    View c0, c1;   // children (even / odd rows), any strides
    int R2, C;
    int i;
    int tiles_x, first_block;
    int ntaps;     // prototype length (4, 6 or 8)
    int stream;    // the plane's stream (Bases::act), -1: none
};

constexpr int DFBA_TILE = 64, DFBA_HALO = 12;   // the halo of the 4-tap prototype (4 (NT - 1) in general)
constexpr int DFBB_ROWS = 16, DFBB_COLS = 120;  // columns of the 4-tap prototype ((128 - 2 (NT - 1)) & ~3 in general)
constexpr int dfbb_cols(int ntaps) { return (128 - 2 * (ntaps - 1)) & ~3; }
constexpr int DFBB_THREADS = 128;        // row-split blocks: four warps, one run of rows each in the ladder passes
constexpr int DFBB_THREADS_WIDE = 256;   // eight warps: for launches smaller than a wave (latency)

// One Laplacian-pyramid tile job (one level of one plane):
//   analysis:  cout = down(main, fa);           out = main - up(cout, fs)
//   synthesis: v = cin - down(main, fa);        out = main + up(v, fs)
// A synthesis job may carry the low-order halves of cin and out (float-float
// lowpass images between the levels; b < 0: absent, the value is cin alone).
struct LpJob {
    View main, cin, cout, out;  // rs = row pitch, cs = 1
    View cin_lo, out_lo;        // synthesis only: low-order parts of cin / out
    int H, W;                   // full-resolution size of this level
    int tiles_x;
    int first_block;
    int stream;                 // the plane's stream (Bases::act), -1: none
    int pad;
};

constexpr int LP_TILE = 64;  // full-resolution output tile edge

// ------------------------------------------------------------- host layout
struct SubbandG {
    long long off;
    int h, w, level, dir, kind;
};
struct PlaneLayout {
    int H, W, L, k[CVC_MAX_LEVELS];
    std::vector<SubbandG> sb;  // lowpass first
    long long total;
};
int modulus(int L, const int* k);
bool make_layout(int H, int W, int L, const int* k, PlaneLayout* out);

// ----------------------------------------------------- transform engine
// A transform plan over a list of planes that share one launch sequence.
struct PlaneRef {
    int H, W, L, k[CVC_MAX_LEVELS];
    View in;          // plane for forward / inverse-adjoint input (rs = pitch), or output for inverse
    long long coef;   // coefficient block offset in B_COEF
    long long work;   // workspace offset in B_WORK
    long long low_coef;   // >= 0: the lowpass lives here instead of at coef (a sub-pyramid of a
                          // larger layout keeps its lowpass apart from its subbands)
    int taps;             // DFB prototype length: 0 or 4, 6 or 8
    int stream;           // the codec stream the plane belongs to (Bases::act), -1: none
};

struct LaunchLp {
    int njobs, nblocks;
    LpJob* d_jobs;
    int* d_block_job;
    int centred;   // level 1 of the forward transform or the inverse: centred single precision
};
struct LaunchDfb {
    int kind;  // 0: DfbAJob, 1: DfbBJob
    int njobs, nblocks;
    void* d_jobs;
    int* d_block_job;
    int ntaps;  // the prototype length of the launch's planes (4, 6 or 8)
};

// Pyramid tail: the coarse levels of a plane whose working images fit in one
// block's shared memory (§2.1 "where the data fits") run in one block of one
// launch: the LP level jobs and the DFB stage jobs of those levels, the same
// tile computations as the per-level launches, executed one after the other
// with the intermediate images resident in shared memory (base B_SMEM); only
// the level's input lowpass (analysis) or output lowpass (synthesis) and the
// coefficients go through global memory.
struct TailStep {
    int kind;     // 0: LpJob, 1: DfbAJob, 2: DfbBJob
    int job;      // index into the launch's table of that kind
    int centred;  // an LP step of the first level (forward or inverse): centred single precision
};
struct TailPlane {
    int first_step, nsteps;
    int ws_floats;  // resident workspace of the plane's levels (floats of shared memory)
    int stream;     // Bases::act
};
struct LaunchTail {
    int nplanes = 0;   // one block each
    int ntaps = 4;
    int ws_floats = 0; // largest resident workspace of the launch's planes
    TailPlane* d_planes = nullptr;
    TailStep* d_steps = nullptr;
    LpJob* d_lp = nullptr;
    DfbAJob* d_a = nullptr;
    DfbBJob* d_b = nullptr;
};
struct TailTables {   // host copy of a tail launch's tables
    int ntaps = 4;
    std::vector<TailPlane> planes;
    std::vector<TailStep> steps;
    std::vector<LpJob> lp;
    std::vector<DfbAJob> a;
    std::vector<DfbBJob> b;
};

enum Mode { FWD = 0, INV = 1, FWD_ADJ = 2, INV_ADJ = 3 };

struct CtEngine {
    std::vector<PlaneRef> planes;
    long long work_elems = 0;
    // per mode: LP launches in execution order and DFB passes in execution order
    std::vector<LaunchLp> lp[4];
    std::vector<LaunchDfb> dfb[4];
    // host copies of the job tables, launch by launch (for plan self-checks)
    std::vector<std::vector<LpJob>> h_lp[4];
    std::vector<std::vector<uint8_t>> h_dfb[4];
    // pyramid-tail launches (forward and inverse only), one per prototype length
    std::vector<LaunchTail> tail[4];
    std::vector<TailTables> h_tail[4];
    // fusion depth: the most coarse levels of a plane that run in its tail (0: none, the
    // default: on B300 one block per plane is slower than the coarse levels' own launches
    // for 1080p planes; the autotuner tries the others); a plane's tail takes as many of
    // them as fit the shared-memory budget
    int tail_levels = 0;
    int dfbb_threads = 0;   // threads per block of the row-split DFB launches (launch_dfb's bthreads)
    std::vector<void*> allocs;
    ~CtEngine();
};

// Build the job tables of all four modes for the given planes.  Workspace
// offsets are assigned by the engine; returns false on allocation failure.
bool engine_build(CtEngine* e, const std::vector<PlaneRef>& planes, bool to_device = true);
size_t workspace_elems(int H, int W, int L);
// the whole transform of mode m (counted in the launch counter)
cudaError_t engine_run(const CtEngine* e, Mode m, Bases bases, cudaStream_t st);
// one part of a mode's launch sequence: part 0 = LP levels, part 1 = DFB passes,
// part 2 = pyramid tails (not counted: the caller adds engine_part_launches).  The tails
// depend on the LP levels in the analysis direction and the LP levels on the tails in
// the synthesis direction; the DFB passes of the other levels are independent of them.
cudaError_t engine_run_part(const CtEngine* e, Mode m, int part, Bases bases, cudaStream_t st);
int engine_part_launches(const CtEngine* e, Mode m, int part);

// process-wide count of kernels launched by the library
void note_launches(long long n);

// -------------------------------------------------------------- kernels
cudaError_t launch_lp(const LaunchLp& L, Mode m, Bases bases, cudaStream_t st);
// one-time kernel attributes of the LP kernels (call before any stream capture)
cudaError_t lp_prepare();
// bthreads: threads per block of the row-split launches (128 or 256; 0: 256 for a launch of
// less than a wave of 128-thread blocks, else 128); it changes no result
cudaError_t launch_dfb(const LaunchDfb& L, Mode m, Bases bases, cudaStream_t st, int bthreads = 0);
// one-time kernel attributes of the DFB kernels (call before any stream capture)
cudaError_t dfb_prepare();
PassParams pass_params(Mode m);
// pyramid tail: shared-memory floats a tail block has for its resident workspace
// (beyond the tile scratch), the launch, and its one-time attributes
int tail_ws_budget(int ntaps);
cudaError_t launch_tail(const LaunchTail& L, Mode m, Bases bases, cudaStream_t st);
cudaError_t tail_prepare();

}  // namespace cvc
