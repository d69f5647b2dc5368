// ct_engine.cu -- coefficient layout and the launch plan of the contourlet
// transform (§2.1, §3.3) over a list of planes.
//
// The transform of every plane is a fixed sequence of steps; the engine
// turns them into job tables once, so that each launch covers one step for
// all planes (and all pyramid levels / DFB channels that take part in it):
//   analysis direction (forward A, adjoint of the inverse S^T):
//     LP level 1 .. L (one launch each), then DFB stage 1 .. kmax (two passes each)
//   synthesis direction (inverse S, adjoint of the forward A^T):
//     DFB stage kmax .. 1 (two passes each), then LP level L .. 1
// Memory is addressed by (base id, offset) so the tables stay valid for any
// input / output pointers.
//
// Directional filter bank reading (§2.1: 2^l wedge subbands, perfect
// reconstruction, ladder fan filters).  A stage splits a channel whose
// samples are o + b1*p1 + b2*p2 into the cosets p1+p2 even / odd with the
// fan prototype betat = (-1, -9, 9, 1)/16 (the 4-tap half-band
// (-1, 9, 9, -1)/16 modulated to the fan):
//   predict (odd):  y = x/2 - (1/2) sum w x[p + delta],   update (even): y = x + sum w y[p + delta]
//   w = betat[a] betat[b],  delta(a,b) = ((a+b)/2, (a-b)/2),  a, b in {-3,-1,1,3}.
// Stage 1 uses b1 = (1,0), b2 = (0,1); its even coset carries the fan
// |w_c| > |w_r| (family "c"), the odd one |w_r| > |w_c| (family "r").
// Stage 2: family c in b1 = (1,1), b2 = (1,-1); family r in (1,1), (-1,1).
// Stage s >= 3, for a channel covering slopes [i/2^m, (i+1)/2^m]:
//   c: b1 = (2^(s-2), -2i), b2 = (2^(s-2), -2i-2);  r: b1 = (-2i, 2^(s-2)), b2 = (-2i-2, 2^(s-2)).
// In the rectangular arrays the channels occupy from stage 3 on (rows
// strided by 2^(s-2), columns by 2 for family c; transposed for r) this is
// a split into even / odd rows (columns) with a 4 x 4 stencil whose rows
// (columns) are sheared by -i per row step: row offset a, column offset
// -i*a + (b-a)/2.  The even child takes the lower half of the slopes.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "cvc_internal.cuh"

namespace cvc {

int modulus(int L, const int* k) {
    int m = 1 << L;
    for (int j = 1; j <= L; j++) {
        int need = (1 << (j - 1)) * (k[j - 1] >= 2 ? (1 << (k[j - 1] - 1)) : 2);
        m = std::max(m, need);
    }
    return m;
}

bool make_layout(int H, int W, int L, const int* k, PlaneLayout* out) {
    if (L < 1 || L > CVC_MAX_LEVELS || H <= 0 || W <= 0) return false;
    for (int j = 0; j < L; j++)
        if (k[j] < 0 || k[j] > CVC_MAX_DIRS_LOG2) return false;
    int M = modulus(L, k);
    if (H % M || W % M) return false;
    out->H = H;
    out->W = W;
    out->L = L;
    for (int j = 0; j < CVC_MAX_LEVELS; j++) out->k[j] = j < L ? k[j] : 0;
    out->sb.clear();
    long long off = 0;
    out->sb.push_back({0, H >> L, W >> L, 0, 0, 0});
    off += (long long)(H >> L) * (W >> L);
    for (int j = 1; j <= L; j++) {
        int hj = H >> (j - 1), wj = W >> (j - 1), kj = k[j - 1], n = 1 << kj;
        for (int d = 0; d < n; d++) {
            SubbandG s{off, 0, 0, j, d, 0};
            if (kj == 0) { s.h = hj; s.w = wj; s.kind = 3; }
            else if (kj == 1) { s.h = hj; s.w = wj / 2; s.kind = 4; }
            else if (d < n / 2) { s.h = hj >> (kj - 1); s.w = wj / 2; s.kind = 1; }
            else { s.h = hj / 2; s.w = wj >> (kj - 1); s.kind = 2; }
            off += (long long)s.h * s.w;
            out->sb.push_back(s);
        }
    }
    out->total = off;
    return true;
}

size_t workspace_elems(int H, int W, int L) {
    size_t n = 0;
    for (int j = 1; j <= L; j++) {
        size_t hj = (size_t)(H >> (j - 1)), wj = (size_t)(W >> (j - 1));
        n += hj * wj + (hj / 2) * (wj / 2);
    }
    return n;
}

CtEngine::~CtEngine() {
    for (void* p : allocs) cudaFree(p);
}

namespace {

const int A4[4] = {-3, -1, 1, 3};
const float BT4[4] = {-1.f / 16, -9.f / 16, 9.f / 16, 1.f / 16};

inline int floordiv2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

struct LiftSpec {     // one pass-independent description of a target coset
    View parent;      // target coset inside the parent (in place)
    View child;       // where the child (output coset) lives after the stage
    int rows, cols;
    int tsel_src;     // unused
};

// Stencil of a target coset: 16 (sel, dr, dc, w)
struct Stencil {
    int8_t sel[16];
    int16_t dr[16], dc[16];
    float w[16];
};

// stage 1 / 2 stencils on polyphase components: target component (pr, pc),
// grid offsets (al, ga) per tap; the source component list is given.
Stencil poly_stencil(int pr, int pc, const int (*off)[2], const int (*srcs)[2], int nsrc) {
    Stencil S;
    int t = 0;
    for (int ia = 0; ia < 4; ia++)
        for (int ib = 0; ib < 4; ib++, t++) {
            int al = off[t][0], ga = off[t][1];
            int qr = (pr + al) & 1, qc = (pc + ga) & 1;
            int sel = -1;
            for (int s = 0; s < nsrc; s++)
                if (srcs[s][0] == qr && srcs[s][1] == qc) sel = s;
            if (sel < 0) { fprintf(stderr, "cvc: internal stencil error\n"); abort(); }
            S.sel[t] = (int8_t)sel;
            S.dr[t] = (int16_t)floordiv2(pr + al);
            S.dc[t] = (int16_t)floordiv2(pc + ga);
            S.w[t] = BT4[ia] * BT4[ib];
        }
    return S;
}

// stage >= 3 stencil; fam 0: split rows, fam 1: split columns; odd target or even target
Stencil shear_stencil(int fam, int i, bool odd_target) {
    Stencil S;
    int t = 0;
    for (int ia = 0; ia < 4; ia++)
        for (int ib = 0; ib < 4; ib++, t++) {
            int a = A4[ia], b = A4[ib];
            int along = odd_target ? (a + 1) / 2 : (a - 1) / 2;  // a odd: exact
            int across = -i * a + (b - a) / 2;
            S.sel[t] = 0;
            if (fam == 0) { S.dr[t] = (int16_t)along; S.dc[t] = (int16_t)across; }
            else { S.dr[t] = (int16_t)across; S.dc[t] = (int16_t)along; }
            S.w[t] = BT4[ia] * BT4[ib];
        }
    return S;
}

View mk(int b, long long off, int rs, int cs) {
    View v;
    v.off = off;
    v.b = b;
    v.rs = rs;
    v.cs = cs;
    return v;
}

// A coset target of one stage: its parent-array view, the view its child
// occupies after the stage, its size and the stencils for both parities.
struct Target {
    View par, chi;
    int rows, cols;
    Stencil st;
    View src_par[2], src_chi[2];  // source coset views before / after the stage
    int nsrc;
};

// All targets of one stage of one (plane, level): odd-parity list and even-parity list
struct StagePlan {
    std::vector<Target> odd, even;
};

struct Chan {
    int T, i;   // family (0 = c, 1 = r), slope index
    View v;     // channel array view (in the detail buffer, or a coefficient slot if final)
    int rows, cols;
};

// Build the stage plans of one DFB (plane, level): D = detail view (B_WORK,
// pitch W), slots = coefficient offsets of the 2^k subbands (B_COEF).
std::vector<StagePlan> dfb_stages(View D, int H, int W, int k, const std::vector<long long>& slot) {
    std::vector<StagePlan> out(k + 1);
    if (k == 0) return out;
    const int Wp = D.rs;
    auto comp = [&](int pr, int pc) { return mk(D.b, D.off + (long long)pr * Wp + pc, 2 * Wp, 2); };
    const int h2 = H / 2, w2 = W / 2;
    // ---- stage 1: polyphase components; E = {00, 11}, O = {01, 10}
    {
        int off[16][2];
        int t = 0;
        for (int ia = 0; ia < 4; ia++)
            for (int ib = 0; ib < 4; ib++, t++) {
                off[t][0] = (A4[ia] + A4[ib]) / 2;
                off[t][1] = (A4[ia] - A4[ib]) / 2;
            }
        const int E[2][2] = {{0, 0}, {1, 1}}, O[2][2] = {{0, 1}, {1, 0}};
        // child views: in place, or the two row-compacted quincunx subbands when k == 1
        auto child = [&](int pr, int pc) {
            if (k > 1) return comp(pr, pc);
            bool even = ((pr + pc) & 1) == 0;
            long long base = slot[even ? 0 : 1];
            // row-compacted subband: row r holds the coset's samples of image row r
            return mk(B_COEF, base + (long long)pr * w2, 2 * w2, 1);
        };
        for (int par = 0; par < 2; par++) {
            const int(*tg)[2] = par ? O : E;
            const int(*sr)[2] = par ? E : O;
            for (int c = 0; c < 2; c++) {
                Target T;
                T.par = comp(tg[c][0], tg[c][1]);
                T.chi = child(tg[c][0], tg[c][1]);
                T.rows = h2;
                T.cols = w2;
                T.st = poly_stencil(tg[c][0], tg[c][1], off, sr, 2);
                T.nsrc = 2;
                for (int s = 0; s < 2; s++) {
                    T.src_par[s] = comp(sr[s][0], sr[s][1]);
                    T.src_chi[s] = child(sr[s][0], sr[s][1]);
                }
                (par ? out[1].odd : out[1].even).push_back(T);
            }
        }
    }
    if (k == 1) return out;
    // ---- stage 2: family c on {00 (E), 11 (O)} with grid offsets (a, b);
    //               family r on {10 (E), 01 (O)} with grid offsets (b, a)
    std::vector<Chan> chans;
    {
        auto child2 = [&](int leaf, int pr, int pc) {
            if (k > 2) return comp(pr, pc);
            return mk(B_COEF, slot[leaf], w2, 1);
        };
        const int fams[2][2][2] = {{{0, 0}, {1, 1}}, {{1, 0}, {0, 1}}};  // [fam][E/O][pr,pc]
        for (int fam = 0; fam < 2; fam++) {
            int off[16][2];
            int t = 0;
            for (int ia = 0; ia < 4; ia++)
                for (int ib = 0; ib < 4; ib++, t++) {
                    off[t][0] = fam == 0 ? A4[ia] : A4[ib];
                    off[t][1] = fam == 0 ? A4[ib] : A4[ia];
                }
            for (int par = 0; par < 2; par++) {
                int pr = fams[fam][par][0], pc = fams[fam][par][1];
                int qr = fams[fam][1 - par][0], qc = fams[fam][1 - par][1];
                int srcs[1][2] = {{qr, qc}};
                Target T;
                T.par = comp(pr, pc);
                T.chi = child2(2 * fam + par, pr, pc);
                T.rows = h2;
                T.cols = w2;
                T.st = poly_stencil(pr, pc, off, srcs, 1);
                T.nsrc = 1;
                T.src_par[0] = comp(qr, qc);
                T.src_chi[0] = child2(2 * fam + (1 - par), qr, qc);
                T.src_par[1] = T.src_par[0];
                T.src_chi[1] = T.src_chi[0];
                (par ? out[2].odd : out[2].even).push_back(T);
            }
            chans.push_back({fam, -1, comp(fams[fam][0][0], fams[fam][0][1]), h2, w2});
            chans.push_back({fam, 0, comp(fams[fam][1][0], fams[fam][1][1]), h2, w2});
        }
    }
    // ---- stages 3..k: even / odd rows (family c) or columns (family r)
    for (int s = 3; s <= k; s++) {
        std::vector<Chan> next;
        const bool fin = (s == k);
        for (size_t ci = 0; ci < chans.size(); ci++) {
            const Chan& C = chans[ci];
            View pe, po;
            int rows = C.rows, cols = C.cols;
            if (C.T == 0) {
                pe = mk(C.v.b, C.v.off, 2 * C.v.rs, C.v.cs);
                po = mk(C.v.b, C.v.off + C.v.rs, 2 * C.v.rs, C.v.cs);
                rows /= 2;
            } else {
                pe = mk(C.v.b, C.v.off, C.v.rs, 2 * C.v.cs);
                po = mk(C.v.b, C.v.off + C.v.cs, C.v.rs, 2 * C.v.cs);
                cols /= 2;
            }
            View ce = pe, co = po;
            if (fin) {
                ce = mk(B_COEF, slot[2 * ci], cols, 1);
                co = mk(B_COEF, slot[2 * ci + 1], cols, 1);
            }
            Target te, to;
            te.par = pe; te.chi = ce; te.rows = rows; te.cols = cols; te.nsrc = 1;
            te.st = shear_stencil(C.T, C.i, false);
            te.src_par[0] = te.src_par[1] = po;
            te.src_chi[0] = te.src_chi[1] = co;
            to.par = po; to.chi = co; to.rows = rows; to.cols = cols; to.nsrc = 1;
            to.st = shear_stencil(C.T, C.i, true);
            to.src_par[0] = to.src_par[1] = pe;
            to.src_chi[0] = to.src_chi[1] = ce;
            out[s].even.push_back(te);
            out[s].odd.push_back(to);
            next.push_back({C.T, 2 * C.i, ce, rows, cols});
            next.push_back({C.T, 2 * C.i + 1, co, rows, cols});
        }
        chans.swap(next);
    }
    return out;
}

LiftJob make_job(const Target& T, View out, View tin, bool src_after, float alpha, float gamma) {
    LiftJob J;
    memset(&J, 0, sizeof(J));
    J.out = out;
    J.tin = tin;
    J.src[0] = src_after ? T.src_chi[0] : T.src_par[0];
    J.src[1] = src_after ? T.src_chi[1] : T.src_par[1];
    J.rows = T.rows;
    J.cols = T.cols;
    J.alpha = alpha;
    J.gamma = gamma;
    for (int t = 0; t < 16; t++) {
        J.w[t] = T.st.w[t];
        J.sel[t] = T.st.sel[t];
        J.dr[t] = T.st.dr[t];
        J.dc[t] = T.st.dc[t];
    }
    return J;
}

template <class Job>
bool upload(std::vector<Job>& jobs, bool to_device, CtEngine* e, Job** d_jobs, int** d_bj, int* nblocks,
            int (*count)(const Job&)) {
    std::vector<int> bj;
    for (size_t i = 0; i < jobs.size(); i++) {
        jobs[i].first_block = (int)bj.size();
        int n = count(jobs[i]);
        for (int b = 0; b < n; b++) bj.push_back((int)i);
    }
    *nblocks = (int)bj.size();
    *d_jobs = nullptr;
    *d_bj = nullptr;
    if (jobs.empty() || !to_device) return true;
    if (cudaMalloc(d_jobs, sizeof(Job) * jobs.size()) != cudaSuccess) return false;
    e->allocs.push_back(*d_jobs);
    if (cudaMalloc(d_bj, sizeof(int) * bj.size()) != cudaSuccess) return false;
    e->allocs.push_back(*d_bj);
    if (cudaMemcpy(*d_jobs, jobs.data(), sizeof(Job) * jobs.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    if (cudaMemcpy(*d_bj, bj.data(), sizeof(int) * bj.size(), cudaMemcpyHostToDevice) != cudaSuccess) return false;
    return true;
}

int count_lift(const LiftJob& J) { return (int)(((long long)J.rows * J.cols + 255) / 256); }
int count_lp(const LpJob& J) {
    int ty = (J.H + LP_TILE - 1) / LP_TILE, tx = (J.W + LP_TILE - 1) / LP_TILE;
    return ty * tx;
}

}  // namespace

static_assert(sizeof(LiftJob) % 4 == 0, "LiftJob is copied as 32-bit words");

bool engine_build(CtEngine* e, const std::vector<PlaneRef>& planes_in, bool to_device) {
    e->planes = planes_in;
    int Lmax = 0, kmax = 0;
    long long work = 0;
    std::vector<PlaneLayout> lays(e->planes.size());
    for (size_t p = 0; p < e->planes.size(); p++) {
        PlaneRef& P = e->planes[p];
        if (!make_layout(P.H, P.W, P.L, P.k, &lays[p])) return false;
        P.work = work;
        work += (long long)workspace_elems(P.H, P.W, P.L);
        Lmax = std::max(Lmax, P.L);
        for (int j = 0; j < P.L; j++) kmax = std::max(kmax, P.k[j]);
    }
    e->work_elems = work;
    for (int m = 0; m < 4; m++) {
        const bool analysis = (m == FWD || m == INV_ADJ);
        const int spatial_base = analysis ? B_IN : B_OUT;
        // ---- LP jobs per level
        std::vector<std::vector<LpJob>> lpj(Lmax + 1);
        // ---- lifting jobs per (stage, pass)
        std::vector<std::vector<LiftJob>> lj1(kmax + 1), lj2(kmax + 1);
        for (size_t p = 0; p < e->planes.size(); p++) {
            const PlaneRef& P = e->planes[p];
            const PlaneLayout& Ly = lays[p];
            long long w = P.work;
            std::vector<long long> coff(P.L + 1), doff(P.L + 1);
            for (int j = 1; j <= P.L; j++) {
                long long hj = P.H >> (j - 1), wj = P.W >> (j - 1);
                doff[j] = w;
                w += hj * wj;
                coff[j] = w;
                w += (hj / 2) * (wj / 2);
            }
            size_t sbi = 1;
            for (int j = 1; j <= P.L; j++) {
                int hj = P.H >> (j - 1), wj = P.W >> (j - 1), kj = P.k[j - 1];
                std::vector<long long> slots;
                for (int d = 0; d < (1 << kj); d++) slots.push_back(P.coef + Ly.sb[sbi + d].off);
                sbi += (size_t)1 << kj;
                View spatial_prev = (j == 1) ? mk(spatial_base, P.in.off, P.in.rs, 1)
                                             : mk(B_WORK, coff[j - 1], wj, 1);
                View low = (j == P.L) ? mk(B_COEF, P.coef + Ly.sb[0].off, wj / 2, 1) : mk(B_WORK, coff[j], wj / 2, 1);
                View det = (kj == 0) ? mk(B_COEF, slots[0], wj, 1) : mk(B_WORK, doff[j], wj, 1);
                LpJob J;
                memset(&J, 0, sizeof(J));
                J.H = hj;
                J.W = wj;
                J.tiles_x = (wj + LP_TILE - 1) / LP_TILE;
                if (analysis) {
                    J.main = spatial_prev;
                    J.cout = low;
                    J.out = det;
                } else {
                    J.main = det;
                    J.cin = low;
                    J.out = spatial_prev;
                }
                lpj[j].push_back(J);
                if (kj == 0) continue;
                std::vector<StagePlan> sp = dfb_stages(mk(B_WORK, doff[j], wj, 1), hj, wj, kj, slots);
                for (int s = 1; s <= kj; s++) {
                    for (const Target& T : sp[s].odd) {
                        if (m == FWD) lj1[s].push_back(make_job(T, T.chi, T.par, false, 0.5f, -0.5f));
                        if (m == INV_ADJ) lj2[s].push_back(make_job(T, T.chi, T.par, true, 2.f, -1.f));
                        if (m == INV) lj2[s].push_back(make_job(T, T.par, T.chi, false, 2.f, 1.f));
                        if (m == FWD_ADJ) lj1[s].push_back(make_job(T, T.par, T.chi, true, 0.5f, 0.5f));
                    }
                    for (const Target& T : sp[s].even) {
                        if (m == FWD) lj2[s].push_back(make_job(T, T.chi, T.par, true, 1.f, 1.f));
                        if (m == INV_ADJ) lj1[s].push_back(make_job(T, T.chi, T.par, false, 1.f, 1.f));
                        if (m == INV) lj1[s].push_back(make_job(T, T.par, T.chi, true, 1.f, -1.f));
                        if (m == FWD_ADJ) lj2[s].push_back(make_job(T, T.par, T.chi, false, 1.f, -1.f));
                    }
                }
            }
        }
        // Pass sources: in the analysis direction, pass 1 reads the parent's
        // other coset, pass 2 the child written by pass 1.  In the synthesis
        // direction pass 1 reads the other child, pass 2 the parent coset
        // written by pass 1 -- make_job's src_after flag encodes exactly that
        // (it selects the child views when true).
        e->lp[m].clear();
        e->lift[m].clear();
        e->h_lp[m].clear();
        e->h_lift[m].clear();
        auto add_lp = [&](std::vector<LpJob>& v) {
            LaunchLp L{};
            if (!upload<LpJob>(v, to_device, e, &L.d_jobs, &L.d_block_job, &L.nblocks, count_lp)) return false;
            L.njobs = (int)v.size();
            e->lp[m].push_back(L);
            e->h_lp[m].push_back(v);
            return true;
        };
        auto add_lift = [&](std::vector<LiftJob>& v) {
            LaunchLift L{};
            if (!upload<LiftJob>(v, to_device, e, &L.d_jobs, &L.d_block_job, &L.nblocks, count_lift)) return false;
            L.njobs = (int)v.size();
            e->lift[m].push_back(L);
            e->h_lift[m].push_back(v);
            return true;
        };
        if (analysis) {
            for (int j = 1; j <= Lmax; j++)
                if (!add_lp(lpj[j])) return false;
            for (int s = 1; s <= kmax; s++)
                if (!add_lift(lj1[s]) || !add_lift(lj2[s])) return false;
        } else {
            for (int s = kmax; s >= 1; s--)
                if (!add_lift(lj1[s]) || !add_lift(lj2[s])) return false;
            for (int j = Lmax; j >= 1; j--)
                if (!add_lp(lpj[j])) return false;
        }
    }
    return true;
}

cudaError_t engine_run_part(const CtEngine* e, Mode m, int part, Bases bases, cudaStream_t st) {
    cudaError_t err = cudaSuccess;
    if (part == 0) {
        for (const LaunchLp& L : e->lp[m]) {
            if ((err = launch_lp(L, m, bases, st)) != cudaSuccess) return err;
            note_launches(L.nblocks > 0);
        }
    } else {
        for (const LaunchLift& L : e->lift[m]) {
            if ((err = launch_lift(L, m, bases, st)) != cudaSuccess) return err;
            note_launches(L.nblocks > 0);
        }
    }
    return err;
}

int engine_part_launches(const CtEngine* e, Mode m, int part) {
    int n = 0;
    if (part == 0)
        for (const LaunchLp& L : e->lp[m]) n += L.nblocks > 0;
    else
        for (const LaunchLift& L : e->lift[m]) n += L.nblocks > 0;
    return n;
}

cudaError_t engine_run(const CtEngine* e, Mode m, Bases bases, cudaStream_t st) {
    const bool analysis = (m == FWD || m == INV_ADJ);
    cudaError_t err = engine_run_part(e, m, analysis ? 0 : 1, bases, st);
    if (err != cudaSuccess) return err;
    return engine_run_part(e, m, analysis ? 1 : 0, bases, st);
}

}  // namespace cvc
