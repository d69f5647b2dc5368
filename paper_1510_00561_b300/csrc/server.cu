// server.cu -- the continuous-batching request loop (cvc_server_*): sessions
// admitted against a device-memory budget, grouped by parameters into
// shards of slots, each shard a multi-stream core replaying its step graph on
// its own CUDA stream.  Host code only; every step runs in the codec kernels.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "codec_core.cuh"

using namespace cvc;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    int kind;
    cvc_batch_io io;
    uint64_t tag;
    int64_t t_submit;
};

enum SessionState { S_WAITING, S_ACTIVE, S_DONE };

struct Session {
    cvc_params prm;
    int state = S_WAITING;
    bool closing = false;
    int shard = -1, slot = -1;
    std::deque<Request> q;
    bool inflight = false;
};

struct Shard {
    Core core;
    cvc_params prm;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    int mode = 0;
    int64_t t_launch = 0;
    std::vector<int> slot_session;   // -1: free
    std::vector<Request> inflight;   // kind 0: none
    size_t bytes = 0;
    int live() const {
        int n = 0;
        for (int s : slot_session) n += s >= 0;
        return n;
    }
    ~Shard() {
        if (ev) cudaEventDestroy(ev);
        if (st) cudaStreamDestroy(st);
    }
};

bool same_params(const cvc_params& a, const cvc_params& b) { return memcmp(&a, &b, sizeof(a)) == 0; }

StreamIo stream_io(const Request& r) {
    StreamIo io{nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0};
    if (r.kind & 1) {
        io.rgb = r.io.d_rgb;
        io.pitch = r.io.pitch_bytes;
        io.out = r.io.d_out;
        io.out_cap = r.io.out_cap;
    }
    if (r.kind & 2) {
        io.in = r.io.d_in;
        io.in_len = r.io.in_len;
        io.rgb_out = r.io.d_rgb_out;
        io.pitch_out = r.io.pitch_out;
    }
    return io;
}

}  // namespace

struct cvc_server {
    cvc_server_config cfg{};
    std::vector<Session> sessions;
    std::vector<std::unique_ptr<Shard>> shards;   // null: freed
    std::deque<int> waiting;
    std::vector<std::pair<cvc_params, size_t>> class_bytes;
    size_t used = 0, peak = 0;
    long long steps = 0, requests_done = 0;
    std::deque<cvc_server_completion> done;
    cvc_status sticky = CVC_OK;

    // device bytes of one shard of these parameters (host-only planning, cached)
    cvc_status shard_bytes(const cvc_params& p, size_t* out) {
        for (auto& cb : class_bytes)
            if (same_params(cb.first, p)) {
                *out = cb.second;
                return CVC_OK;
            }
        Core c;
        std::vector<cvc_params> v(cfg.slots_per_shard, p);
        cvc_status s = core_plan(&c, v.data(), cfg.slots_per_shard);
        if (s != CVC_OK) return s;
        *out = core_device_bytes(&c);
        class_bytes.push_back({p, *out});
        return CVC_OK;
    }

    void complete(Shard* sh, int slot, cvc_status fail) {
        Request& r = sh->inflight[slot];
        cvc_server_completion cpl;
        memset(&cpl, 0, sizeof(cpl));
        cpl.tag = r.tag;
        cpl.session = sh->slot_session[slot];
        cpl.kind = r.kind;
        cpl.frame_type = cpl.dec_frame_type = -1;
        if (fail == CVC_OK) {
            unsigned didx = 0;
            core_commit(&sh->core, slot, sh->mode, &cpl.enc_status, &cpl.dec_status, &cpl.out_len, &cpl.frame_type,
                        &cpl.dec_frame_type, &didx);
        } else {
            cpl.enc_status = (r.kind & 1) ? fail : CVC_OK;
            cpl.dec_status = (r.kind & 2) ? fail : CVC_OK;
        }
        cpl.t_submit_ns = r.t_submit;
        cpl.t_launch_ns = sh->t_launch;
        cpl.t_done_ns = now_ns();
        done.push_back(cpl);
        requests_done++;
        r.kind = 0;
        sessions[cpl.session].inflight = false;
    }

    // collect finished steps; returns the number of shards that finished
    int reap() {
        int n = 0;
        for (auto& up : shards) {
            Shard* sh = up.get();
            if (!sh || !sh->busy) continue;
            cudaError_t q = cudaEventQuery(sh->ev);
            if (q == cudaErrorNotReady) continue;
            cvc_status fail = CVC_OK;
            if (q != cudaSuccess) {
                cudaGetLastError();
                fail = CVC_ERR_CUDA;
                sticky = CVC_ERR_CUDA;
            }
            for (int s = 0; s < (int)sh->inflight.size(); s++)
                if (sh->inflight[s].kind) complete(sh, s, fail);
            sh->busy = false;
            n++;
        }
        return n;
    }

    void retire() {
        for (int id = 0; id < (int)sessions.size(); id++) {
            Session& S = sessions[id];
            if (S.state == S_DONE || !S.closing || !S.q.empty() || S.inflight) continue;
            if (S.state == S_WAITING) {
                waiting.erase(std::remove(waiting.begin(), waiting.end(), id), waiting.end());
            } else {
                shards[S.shard]->slot_session[S.slot] = -1;
            }
            S.state = S_DONE;
        }
        for (auto& up : shards) {
            if (!up || up->busy || up->live() > 0) continue;
            used -= up->bytes;
            up.reset();
        }
    }

    bool create_shard(const cvc_params& p, size_t bytes, int* index) {
        std::unique_ptr<Shard> sh(new (std::nothrow) Shard());
        if (!sh) return false;
        std::vector<cvc_params> v(cfg.slots_per_shard, p);
        if (core_plan(&sh->core, v.data(), cfg.slots_per_shard) != CVC_OK || core_alloc(&sh->core) != CVC_OK)
            return false;
        for (int m = STEP_ENC; m <= STEP_ENCDEC; m++)
            if (core_capture(&sh->core, m) != CVC_OK) return false;
        if (cudaStreamCreateWithFlags(&sh->st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sh->ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        sh->prm = p;
        sh->bytes = bytes;
        sh->slot_session.assign(cfg.slots_per_shard, -1);
        sh->inflight.assign(cfg.slots_per_shard, Request{0, {}, 0, 0});
        for (size_t i = 0; i < shards.size(); i++)
            if (!shards[i]) {
                shards[i] = std::move(sh);
                *index = (int)i;
                return true;
            }
        shards.push_back(std::move(sh));
        *index = (int)shards.size() - 1;
        return true;
    }

    // first fit in opening order
    void admit() {
        for (auto it = waiting.begin(); it != waiting.end();) {
            Session& S = sessions[*it];
            int where = -1, slot = -1;
            for (size_t i = 0; i < shards.size() && where < 0; i++) {
                Shard* sh = shards[i].get();
                if (!sh || !same_params(sh->prm, S.prm)) continue;
                for (int s = 0; s < (int)sh->slot_session.size(); s++)
                    if (sh->slot_session[s] < 0 && !sh->inflight[s].kind) {
                        where = (int)i;
                        slot = s;
                        break;
                    }
            }
            if (where < 0) {
                size_t bytes = 0;
                if (shard_bytes(S.prm, &bytes) == CVC_OK && used + bytes <= cfg.budget_bytes &&
                    create_shard(S.prm, bytes, &where)) {
                    used += bytes;
                    peak = std::max(peak, used);
                    slot = 0;
                }
            }
            if (where < 0) {
                ++it;
                continue;
            }
            Shard* sh = shards[where].get();
            sh->slot_session[slot] = *it;
            core_reset(&sh->core, slot);
            S.state = S_ACTIVE;
            S.shard = where;
            S.slot = slot;
            it = waiting.erase(it);
        }
    }

    void launch() {
        for (auto& up : shards) {
            Shard* sh = up.get();
            if (!sh || sh->busy) continue;
            int mode = 0;
            for (int s = 0; s < (int)sh->slot_session.size(); s++) {
                const int id = sh->slot_session[s];
                if (id < 0) continue;
                Session& S = sessions[id];
                if (S.q.empty() || S.inflight) continue;
                sh->inflight[s] = S.q.front();
                S.q.pop_front();
                S.inflight = true;
                mode |= sh->inflight[s].kind;
            }
            if (!mode) continue;
            const StreamIo none{nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0};
            cvc_status st = core_begin(&sh->core) ? CVC_OK : CVC_ERR_CUDA;
            for (int s = 0; s < (int)sh->slot_session.size() && st == CVC_OK; s++)
                core_fill_call(&sh->core, s, mode, sh->inflight[s].kind ? stream_io(sh->inflight[s]) : none);
            sh->mode = mode;
            sh->t_launch = now_ns();
            if (st == CVC_OK) st = core_enqueue(&sh->core, mode, sh->st);
            if (st == CVC_OK && cudaEventRecord(sh->ev, sh->st) != cudaSuccess) st = CVC_ERR_CUDA;
            if (st != CVC_OK) {
                cudaGetLastError();
                sticky = st;
                for (int s = 0; s < (int)sh->inflight.size(); s++)
                    if (sh->inflight[s].kind) complete(sh, s, st);
                continue;
            }
            sh->busy = true;
            steps++;
        }
    }

    bool any_busy() const {
        for (auto& up : shards)
            if (up && up->busy) return true;
        return false;
    }

    void cycle() {
        reap();
        retire();
        admit();
        launch();
    }
};

extern "C" {

int64_t cvc_server_now_ns(void) { return now_ns(); }

cvc_status cvc_server_create(const cvc_server_config* cfg, cvc_server** out) {
    if (!out) return CVC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || cfg->slots_per_shard < 1 || cfg->slots_per_shard > 256 || cfg->budget_bytes == 0)
        return CVC_ERR_INVALID_ARG;
    cvc_server* s = new (std::nothrow) cvc_server();
    if (!s) return CVC_ERR_NOMEM;
    s->cfg = *cfg;
    *out = s;
    return CVC_OK;
}

cvc_status cvc_server_destroy(cvc_server* s) {
    if (!s) return CVC_OK;
    for (auto& up : s->shards)
        if (up && up->busy) cudaEventSynchronize(up->ev);
    delete s;
    return CVC_OK;
}

cvc_status cvc_server_open(cvc_server* s, const cvc_params* params, int* session) {
    if (!s || !params || !session) return CVC_ERR_INVALID_ARG;
    if (!codec_params_valid(params)) return CVC_ERR_INVALID_ARG;
    if (params->chroma_420 != 1) return CVC_ERR_UNSUPPORTED;
    size_t bytes = 0;
    cvc_status st = s->shard_bytes(*params, &bytes);
    if (st != CVC_OK) return st;
    if (bytes > s->cfg.budget_bytes) return CVC_ERR_NOMEM;
    Session S;
    S.prm = *params;
    s->sessions.push_back(S);
    *session = (int)s->sessions.size() - 1;
    s->waiting.push_back(*session);
    s->admit();
    return CVC_OK;
}

cvc_status cvc_server_close(cvc_server* s, int session) {
    if (!s || session < 0 || session >= (int)s->sessions.size() || s->sessions[session].state == S_DONE)
        return CVC_ERR_INVALID_ARG;
    s->sessions[session].closing = true;
    return CVC_OK;
}

cvc_status cvc_server_submit(cvc_server* s, int session, int kind, const cvc_batch_io* io, uint64_t tag) {
    if (!s || !io || session < 0 || session >= (int)s->sessions.size() || kind < 1 || kind > 3)
        return CVC_ERR_INVALID_ARG;
    Session& S = s->sessions[session];
    if (S.closing || S.state == S_DONE) return CVC_ERR_INVALID_ARG;
    const size_t row = (size_t)S.prm.width * 3;
    if ((kind & 1) && (!io->d_rgb || io->pitch_bytes < row || !io->d_out || ((uintptr_t)io->d_out & 3)))
        return CVC_ERR_INVALID_ARG;
    if ((kind & 2) && (!io->d_rgb_out || io->pitch_out < row || (kind == 2 && !io->d_in)))
        return CVC_ERR_INVALID_ARG;
    S.q.push_back(Request{kind, *io, tag, now_ns()});
    return CVC_OK;
}

cvc_status cvc_server_poll(cvc_server* s, int wait_us, cvc_server_completion* out, int max_out, int* n_out) {
    if (!s || (max_out > 0 && !out)) return CVC_ERR_INVALID_ARG;
    s->cycle();
    if (s->done.empty() && wait_us > 0) {
        const int64_t deadline = now_ns() + (int64_t)wait_us * 1000;
        // spin (yielding) on the shards' events until one finishes or the wait ends
        while (s->any_busy() && s->done.empty() && now_ns() < deadline) {
            std::this_thread::yield();
            s->cycle();
        }
    }
    int n = 0;
    while (n < max_out && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    if (n_out) *n_out = n;
    cvc_status st = s->sticky;
    s->sticky = CVC_OK;
    return st;
}

cvc_status cvc_server_get_stats(const cvc_server* s, cvc_server_stats* out) {
    if (!s || !out) return CVC_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->budget_bytes = s->cfg.budget_bytes;
    out->used_bytes = s->used;
    out->peak_used_bytes = s->peak;
    for (auto& up : s->shards) out->shards += up != nullptr;
    long long queued = 0;
    for (const Session& S : s->sessions) {
        out->active_sessions += S.state == S_ACTIVE;
        out->waiting_sessions += S.state == S_WAITING;
        queued += (long long)S.q.size();
    }
    out->steps = s->steps;
    out->requests_done = s->requests_done;
    out->requests_queued = queued;
    return CVC_OK;
}

}  // extern "C"
