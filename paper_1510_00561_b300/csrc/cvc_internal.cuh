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
enum { B_IN = 0, B_COEF = 1, B_WORK = 2, B_OUT = 3, N_BASES = 4 };
struct Bases {
    float* p[N_BASES];
};

// Strided 2-D view: element (u, v) is at base[b] + off + u*rs + v*cs.
struct View {
    long long off;
    int b;
    int rs, cs;
};

// One lifting pass of the directional filter bank on one target coset array:
//   out(u,v) = alpha * tin(u,v) + gamma * sum_t w[t] * src_{sel[t]}((u+dr[t]) mod rows, (v+dc[t]) mod cols)
struct LiftJob {
    View out, tin, src[2];
    int rows, cols;
    float alpha, gamma;
    float w[16];
    int8_t sel[16];
    int16_t dr[16], dc[16];
    int first_block;  // first flat block of this job in the launch
};

// One Laplacian-pyramid tile job (one level of one plane):
//   analysis:  cout = down(main, fa);           out = main - up(cout, fs)
//   synthesis: v = cin - down(main, fa);        out = main + up(v, fs)
struct LpJob {
    View main, cin, cout, out;  // rs = row pitch, cs = 1
    int H, W;                   // full-resolution size of this level
    int tiles_x;
    int first_block;
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
};

struct LaunchLp {
    int njobs, nblocks;
    LpJob* d_jobs;
    int* d_block_job;
};
struct LaunchLift {
    int njobs, nblocks;
    LiftJob* d_jobs;
    int* d_block_job;
};

enum Mode { FWD = 0, INV = 1, FWD_ADJ = 2, INV_ADJ = 3 };

struct CtEngine {
    std::vector<PlaneRef> planes;
    long long work_elems = 0;
    // per mode: LP launches in execution order and DFB passes in execution order
    std::vector<LaunchLp> lp[4];
    std::vector<LaunchLift> lift[4];
    // host copies of the job tables, launch by launch (for plan self-checks)
    std::vector<std::vector<LpJob>> h_lp[4];
    std::vector<std::vector<LiftJob>> h_lift[4];
    std::vector<void*> allocs;
    ~CtEngine();
};

// Build the job tables of all four modes for the given planes.  Workspace
// offsets are assigned by the engine; returns false on allocation failure.
bool engine_build(CtEngine* e, const std::vector<PlaneRef>& planes, bool to_device = true);
size_t workspace_elems(int H, int W, int L);
cudaError_t engine_run(const CtEngine* e, Mode m, Bases bases, cudaStream_t st);
// one part of a mode's launch sequence: part 0 = LP levels, part 1 = DFB passes
cudaError_t engine_run_part(const CtEngine* e, Mode m, int part, Bases bases, cudaStream_t st);
int engine_part_launches(const CtEngine* e, Mode m, int part);

// process-wide count of kernels launched by the library
void note_launches(int n);

// -------------------------------------------------------------- kernels
cudaError_t launch_lp(const LaunchLp& L, Mode m, Bases bases, cudaStream_t st);
cudaError_t launch_lift(const LaunchLift& L, Mode m, Bases bases, cudaStream_t st);

}  // namespace cvc
