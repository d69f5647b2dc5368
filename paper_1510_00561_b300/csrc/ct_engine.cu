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
// The even child takes the lower half of the slopes.
//
// Longer prototypes (6 or 8 taps, PlaneRef.taps) take the same tile kernels
// instantiated for their length; planes of different lengths get separate
// launches of each step.
//
// Data flow of one level: the LP writes the detail image D; stages 1 and 2
// run fused in k_dfb_a, whose stage-2 channels are D's four polyphase
// classes; from stage 3 on every channel is a compact array, and a stage is a
// split of it into even / odd rows with a 4 x 4 stencil whose columns shear by
// -i per row (row offset a, column offset -i*a + (b-a)/2), run by k_dfb_b.
// Family-r channels are stored transposed between stages so that the same row
// split serves them; the last stage writes every subband into its slot of the
// coefficient layout (family r transposed back).  Channels of a stage sit in
// tree order, channel c at offset c * H*W / 2^(s-1) of a ping-pong pair of
// level buffers.
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
        n += 2 * hj * wj + (hj / 2) * (wj / 2);   // detail D_j, its ping-pong partner Q_j, lowpass c_j
    }
    return n;
}

CtEngine::~CtEngine() {
    for (void* p : allocs) cudaFree(p);
}

namespace {

View mk(int b, long long off, int rs, int cs) {
    View v;
    v.off = off;
    v.b = b;
    v.rs = rs;
    v.cs = cs;
    return v;
}

// DFB jobs of one (plane, level): detail D_j at doff, partner Q_j at qoff,
// subband slots (coefficient offsets) in tree order.
void dfb_jobs(int H, int W, int k, int ntaps, int stream, int wb, long long doff, long long qoff,
              const std::vector<long long>& slot, std::vector<DfbAJob>& ajobs,
              std::vector<std::vector<DfbBJob>>& bjobs) {
    if (k == 0) return;
    const int h2 = H / 2, w2 = W / 2;
    const long long hw = (long long)H * W;
    DfbAJob A;
    memset(&A, 0, sizeof(A));
    A.D = mk(wb, doff, W, 1);
    A.H = H;
    A.W = W;
    A.nst = k == 1 ? 1 : 2;
    A.tiles_x = (W + DFBA_TILE - 1) / DFBA_TILE;
    A.ntaps = ntaps;
    A.stream = stream;
    // polyphase classes q = 2*pr + pc: 00, 01, 10, 11
    if (k == 1) {
        // stage-1 cosets are the subbands: {00, 11} row-compacted into slot 0, {01, 10} into slot 1
        A.comp[0] = mk(B_COEF, slot[0], W, 1);
        A.comp[3] = mk(B_COEF, slot[0] + w2, W, 1);
        A.comp[1] = mk(B_COEF, slot[1], W, 1);
        A.comp[2] = mk(B_COEF, slot[1] + w2, W, 1);
    } else if (k == 2) {
        // stage-2 channels in tree order: c(i=-1) = 00, c(i=0) = 11, r(i=-1) = 10, r(i=0) = 01
        A.comp[0] = mk(B_COEF, slot[0], w2, 1);
        A.comp[3] = mk(B_COEF, slot[1], w2, 1);
        A.comp[2] = mk(B_COEF, slot[2], w2, 1);
        A.comp[1] = mk(B_COEF, slot[3], w2, 1);
    } else {
        // compact channel arrays in Q_j, family r transposed ((W/2) x (H/2))
        A.comp[0] = mk(wb, qoff, w2, 1);
        A.comp[3] = mk(wb, qoff + hw / 4, w2, 1);
        A.comp[2] = mk(wb, qoff + 2 * hw / 4, 1, h2);
        A.comp[1] = mk(wb, qoff + 3 * hw / 4, 1, h2);
    }
    ajobs.push_back(A);
    if (k <= 2) return;
    // stages 3..k: channel list (family, slope index) in tree order
    std::vector<std::pair<int, int>> ch = {{0, -1}, {0, 0}, {1, -1}, {1, 0}};
    for (int s = 3; s <= k; s++) {
        const bool fin = (s == k);
        const long long xin = (s % 2 == 1) ? qoff : doff;    // stage 3 reads Q_j, writes D_j, ...
        const long long yout = (s % 2 == 1) ? doff : qoff;
        const long long csize = hw >> (s - 1);               // elements of one stage-s channel
        std::vector<std::pair<int, int>> next;
        for (size_t c = 0; c < ch.size(); c++) {
            const int fam = ch[c].first, i = ch[c].second;
            const int R = fam == 0 ? (H >> (s - 2)) : (W >> (s - 2));
            const int C = fam == 0 ? w2 : h2;
            const int R2 = R / 2;
            DfbBJob J;
            memset(&J, 0, sizeof(J));
            const long long off = xin + (long long)c * csize;
            J.pe = mk(wb, off, 2 * C, 1);
            J.po = mk(wb, off + C, 2 * C, 1);
            if (!fin) {
                const long long co = yout + (long long)c * csize;
                J.c0 = mk(wb, co, C, 1);
                J.c1 = mk(wb, co + csize / 2, C, 1);
            } else if (fam == 0) {
                J.c0 = mk(B_COEF, slot[2 * c], C, 1);
                J.c1 = mk(B_COEF, slot[2 * c + 1], C, 1);
            } else {
                // subband (H/2) x (W >> (k-1)) is the transpose of the R2 x C child
                J.c0 = mk(B_COEF, slot[2 * c], 1, R2);
                J.c1 = mk(B_COEF, slot[2 * c + 1], 1, R2);
            }
            J.R2 = R2;
            J.C = C;
            J.i = i;
            J.tiles_x = (C + dfbb_cols(ntaps) - 1) / dfbb_cols(ntaps);
            J.ntaps = ntaps;
            J.stream = stream;
            bjobs[s].push_back(J);
            next.push_back({fam, 2 * i});
            next.push_back({fam, 2 * i + 1});
        }
        ch.swap(next);
    }
}

template <class Job>
bool upload(std::vector<Job>& jobs, bool to_device, CtEngine* e, void** d_jobs, int** d_bj, int* nblocks,
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

int count_lp(const LpJob& J) {
    int ty = (J.H + LP_TILE - 1) / LP_TILE, tx = (J.W + LP_TILE - 1) / LP_TILE;
    return ty * tx;
}
int count_a(const DfbAJob& J) {
    return ((J.H + DFBA_TILE - 1) / DFBA_TILE) * J.tiles_x;
}
int count_b(const DfbBJob& J) {
    return ((J.R2 + DFBB_ROWS - 1) / DFBB_ROWS) * J.tiles_x;
}

// the levels t..L of a plane whose resident workspace (detail, partner and lowpass
// image of each) fits `budget` floats, at most `most` of them; returns t (L + 1: none)
int tail_start(const PlaneRef& P, int most, long long budget) {
    int t = P.L + 1;
    long long ws = 0;
    for (int j = P.L; j >= 1 && P.L - j + 1 <= most; j--) {
        const long long hj = P.H >> (j - 1), wj = P.W >> (j - 1);
        ws += 2 * hj * wj + (hj / 2) * (wj / 2);
        if (ws > budget) break;
        t = j;
    }
    return t;
}

bool upload_tail(TailTables& T, bool to_device, CtEngine* e, LaunchTail* L) {
    L->nplanes = (int)T.planes.size();
    L->ntaps = T.ntaps;
    L->ws_floats = 0;
    for (const TailPlane& P : T.planes) L->ws_floats = std::max(L->ws_floats, P.ws_floats);
    if (!to_device || T.planes.empty()) return true;
    auto put = [&](const void* src, size_t bytes, void** dst) {
        if (bytes == 0) return true;
        if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
        e->allocs.push_back(*dst);
        return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    return put(T.planes.data(), sizeof(TailPlane) * T.planes.size(), (void**)&L->d_planes) &&
           put(T.steps.data(), sizeof(TailStep) * T.steps.size(), (void**)&L->d_steps) &&
           put(T.lp.data(), sizeof(LpJob) * T.lp.size(), (void**)&L->d_lp) &&
           put(T.a.data(), sizeof(DfbAJob) * T.a.size(), (void**)&L->d_a) &&
           put(T.b.data(), sizeof(DfbBJob) * T.b.size(), (void**)&L->d_b);
}

}  // namespace

bool engine_build(CtEngine* e, const std::vector<PlaneRef>& planes_in, bool to_device) {
    for (void* p : e->allocs) cudaFree(p);
    e->allocs.clear();
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
        const bool tails = (m == FWD || m == INV) && e->tail_levels > 0;
        const int spatial_base = analysis ? B_IN : B_OUT;
        std::vector<std::vector<LpJob>> lpj(Lmax + 1);
        // tile jobs by prototype length (4, 6, 8): one launch per length and step
        std::vector<DfbAJob> aj[3];
        std::vector<std::vector<DfbBJob>> bj[3];
        for (auto& v : bj) v.resize(std::max(kmax, 2) + 1);
        TailTables tt[3];
        for (int n = 0; n < 3; n++) tt[n].ntaps = 4 + 2 * n;

        for (size_t p = 0; p < e->planes.size(); p++) {
            const PlaneRef& P = e->planes[p];
            const PlaneLayout& Ly = lays[p];
            const int nt = (P.taps == 6 || P.taps == 8) ? P.taps : 4;
            const int t = tails ? tail_start(P, e->tail_levels, tail_ws_budget(nt)) : P.L + 1;
            long long w = P.work;
            std::vector<long long> coff(P.L + 1), doff(P.L + 1), qoff(P.L + 1);
            for (int j = 1; j <= P.L; j++) {
                long long hj = P.H >> (j - 1), wj = P.W >> (j - 1);
                doff[j] = w;
                w += hj * wj;
                qoff[j] = w;
                w += hj * wj;
                coff[j] = w;
                w += (hj / 2) * (wj / 2);
            }
            // the tail's resident workspace: the same layout for levels t..L, from 0
            std::vector<long long> sd(P.L + 1), sq(P.L + 1), scf(P.L + 1);
            long long ws = 0;
            for (int j = t; j <= P.L; j++) {
                long long hj = P.H >> (j - 1), wj = P.W >> (j - 1);
                sd[j] = ws;
                ws += hj * wj;
                sq[j] = ws;
                ws += hj * wj;
                scf[j] = ws;
                ws += (hj / 2) * (wj / 2);
            }
            TailTables& T = tt[nt / 2 - 2];
            TailPlane tp{(int)T.steps.size(), 0, (int)ws, P.stream};
            // the jobs of each level, in the order the tail runs them
            std::vector<std::vector<TailStep>> level_steps(P.L + 1);
            size_t sbi = 1;
            for (int j = 1; j <= P.L; j++) {
                int hj = P.H >> (j - 1), wj = P.W >> (j - 1), kj = P.k[j - 1];
                const bool in_tail = j >= t;
                const int wb = in_tail ? B_SMEM : B_WORK;
                const std::vector<long long>& D = in_tail ? sd : doff;
                const std::vector<long long>& Q = in_tail ? sq : qoff;
                const std::vector<long long>& Cf = in_tail ? scf : coff;
                std::vector<long long> slots;
                for (int d = 0; d < (1 << kj); d++) slots.push_back(P.coef + Ly.sb[sbi + d].off);
                sbi += (size_t)1 << kj;
                // level j's input (analysis) / output (synthesis) image: the plane at level 1, else
                // the lowpass c_{j-1}, resident when level j-1 is in the tail as well
                View spatial_prev = (j == 1) ? mk(spatial_base, P.in.off, P.in.rs, 1)
                                             : (j - 1 >= t ? mk(B_SMEM, scf[j - 1], wj, 1)
                                                           : mk(B_WORK, coff[j - 1], wj, 1));
                const long long low_at = P.low_coef >= 0 ? P.low_coef : P.coef + Ly.sb[0].off;
                View low = (j == P.L) ? mk(B_COEF, low_at, wj / 2, 1) : mk(wb, Cf[j], wj / 2, 1);
                View det = (kj == 0) ? mk(B_COEF, slots[0], wj, 1) : mk(wb, D[j], wj, 1);
                LpJob J;
                memset(&J, 0, sizeof(J));
                J.H = hj;
                J.W = wj;
                J.tiles_x = (wj + LP_TILE - 1) / LP_TILE;
                J.stream = P.stream;
                J.cin_lo = mk(-1, 0, 0, 0);
                J.out_lo = mk(-1, 0, 0, 0);
                if (analysis) {
                    J.main = spatial_prev;
                    J.cout = low;
                    J.out = det;
                } else {
                    J.main = det;
                    J.cin = low;
                    J.out = spatial_prev;
                    // the lowpass images between synthesis levels are float-float: the low-order
                    // part of c_{j-1} (level j's output, hj x wj) goes to Q_j, free once the DFB
                    // synthesis has run; level j reads that of c_j from Q_{j+1} (resident inside
                    // the tail; the tail's last output goes to the global Q_t for level t-1)
                    if (j >= 2) J.out_lo = (j - 1 >= t) ? mk(B_SMEM, sq[j], wj, 1) : mk(B_WORK, qoff[j], wj, 1);
                    if (j < P.L) J.cin_lo = mk(wb, Q[j + 1], wj / 2, 1);
                }
                if (!in_tail) {
                    lpj[j].push_back(J);
                    dfb_jobs(hj, wj, kj, nt, P.stream, B_WORK, doff[j], qoff[j], slots, aj[nt / 2 - 2],
                             bj[nt / 2 - 2]);
                    continue;
                }
                std::vector<DfbAJob> la;
                std::vector<std::vector<DfbBJob>> lb(std::max(kj, 2) + 1);
                dfb_jobs(hj, wj, kj, nt, P.stream, B_SMEM, sd[j], sq[j], slots, la, lb);
                std::vector<TailStep>& st = level_steps[j];
                auto step_lp = [&]() {
                    st.push_back({0, (int)T.lp.size(), (m == FWD || m == INV) && j == 1});
                    T.lp.push_back(J);
                };
                auto step_a = [&]() {
                    for (DfbAJob& A : la) {
                        st.push_back({1, (int)T.a.size(), 0});
                        T.a.push_back(A);
                    }
                };
                auto step_b = [&](int s) {
                    for (DfbBJob& Bj : lb[s]) {
                        st.push_back({2, (int)T.b.size(), 0});
                        T.b.push_back(Bj);
                    }
                };
                if (analysis) {
                    step_lp();
                    step_a();
                    for (int s = 3; s <= kj; s++) step_b(s);
                } else {
                    for (int s = kj; s >= 3; s--) step_b(s);
                    step_a();
                    step_lp();
                }
            }
            if (t <= P.L) {
                // analysis runs levels t..L, synthesis L..t
                for (int j = analysis ? t : P.L; analysis ? j <= P.L : j >= t; j += analysis ? 1 : -1)
                    T.steps.insert(T.steps.end(), level_steps[j].begin(), level_steps[j].end());
                tp.nsteps = (int)T.steps.size() - tp.first_step;
                T.planes.push_back(tp);
            }
        }
        e->lp[m].clear();
        e->dfb[m].clear();
        e->tail[m].clear();
        e->h_lp[m].clear();
        e->h_dfb[m].clear();
        e->h_tail[m].clear();
        // the first level of the forward transform and the inverse runs centred in single precision (k_lp.cu)
        auto add_lp = [&](std::vector<LpJob>& v, bool centred) {
            LaunchLp L{};
            L.centred = centred;
            void* dj = nullptr;
            if (!upload<LpJob>(v, to_device, e, &dj, &L.d_block_job, &L.nblocks, count_lp)) return false;
            L.d_jobs = static_cast<LpJob*>(dj);
            L.njobs = (int)v.size();
            e->lp[m].push_back(L);
            e->h_lp[m].push_back(v);
            return true;
        };
        auto add_a = [&](std::vector<DfbAJob>& v) {
            LaunchDfb L{};
            L.kind = 0;
            L.ntaps = v.front().ntaps;
            if (!upload<DfbAJob>(v, to_device, e, &L.d_jobs, &L.d_block_job, &L.nblocks, count_a)) return false;
            L.njobs = (int)v.size();
            e->dfb[m].push_back(L);
            e->h_dfb[m].emplace_back(reinterpret_cast<uint8_t*>(v.data()),
                                     reinterpret_cast<uint8_t*>(v.data() + v.size()));
            return true;
        };
        auto add_b = [&](std::vector<DfbBJob>& v) {
            LaunchDfb L{};
            L.kind = 1;
            L.ntaps = v.front().ntaps;
            if (!upload<DfbBJob>(v, to_device, e, &L.d_jobs, &L.d_block_job, &L.nblocks, count_b)) return false;
            L.njobs = (int)v.size();
            e->dfb[m].push_back(L);
            e->h_dfb[m].emplace_back(reinterpret_cast<uint8_t*>(v.data()),
                                     reinterpret_cast<uint8_t*>(v.data() + v.size()));
            return true;
        };
        for (int n = 0; n < 3; n++) {
            if (tt[n].planes.empty()) continue;
            LaunchTail L;
            if (!upload_tail(tt[n], to_device, e, &L)) return false;
            e->tail[m].push_back(L);
            e->h_tail[m].push_back(tt[n]);
        }
        if (analysis) {
            for (int j = 1; j <= Lmax; j++)
                if (!add_lp(lpj[j], m == FWD && j == 1)) return false;
            for (int n = 0; n < 3; n++)
                if (!aj[n].empty() && !add_a(aj[n])) return false;
            for (int s = 3; s <= kmax; s++)
                for (int n = 0; n < 3; n++)
                    if (!bj[n][s].empty() && !add_b(bj[n][s])) return false;
        } else {
            for (int s = kmax; s >= 3; s--)
                for (int n = 0; n < 3; n++)
                    if (!bj[n][s].empty() && !add_b(bj[n][s])) return false;
            for (int n = 0; n < 3; n++)
                if (!aj[n].empty() && !add_a(aj[n])) return false;
            for (int j = Lmax; j >= 1; j--)
                if (!add_lp(lpj[j], m == INV && j == 1)) return false;
        }
    }
    return true;
}

cudaError_t engine_run_part(const CtEngine* e, Mode m, int part, Bases bases, cudaStream_t st) {
    cudaError_t err = cudaSuccess;
    if (part == 0) {
        for (const LaunchLp& L : e->lp[m])
            if ((err = launch_lp(L, m, bases, st)) != cudaSuccess) return err;
    } else if (part == 1) {
        for (const LaunchDfb& L : e->dfb[m])
            if ((err = launch_dfb(L, m, bases, st, e->dfbb_threads)) != cudaSuccess) return err;
    } else {
        for (const LaunchTail& L : e->tail[m])
            if ((err = launch_tail(L, m, bases, st)) != cudaSuccess) return err;
    }
    return err;
}

int engine_part_launches(const CtEngine* e, Mode m, int part) {
    int n = 0;
    if (part == 0)
        for (const LaunchLp& L : e->lp[m]) n += L.nblocks > 0;
    else if (part == 1)
        for (const LaunchDfb& L : e->dfb[m]) n += L.nblocks > 0;
    else
        for (const LaunchTail& L : e->tail[m]) n += L.nplanes > 0;
    return n;
}

// everything on one stream: analysis LP levels, tails (they read the last global level's
// lowpass), DFB stages; synthesis DFB stages, tails (they write it), LP levels
cudaError_t engine_run(const CtEngine* e, Mode m, Bases bases, cudaStream_t st) {
    const bool analysis = (m == FWD || m == INV_ADJ);
    const int order[3] = {analysis ? 0 : 1, 2, analysis ? 1 : 0};
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < 3 && err == cudaSuccess; k++) err = engine_run_part(e, m, order[k], bases, st);
    if (err == cudaSuccess)
        note_launches(engine_part_launches(e, m, 0) + engine_part_launches(e, m, 1) + engine_part_launches(e, m, 2));
    return err;
}

}  // namespace cvc
