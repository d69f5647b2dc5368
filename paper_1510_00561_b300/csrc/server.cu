// server.cu -- the continuous-batching request loop (cvc_server_*): sessions
// admitted against a device-memory budget, grouped by parameters into
// shards of slots, each shard a multi-stream core replaying its step graph on
// its own CUDA stream.  A shard keeps up to `depth` steps in flight: requests
// that arrive while a step runs are queued behind it at once (the coder state
// lives on the device, so the next step needs nothing from the host), and
// shards of smaller frames run on higher-priority streams so that their short
// steps do not wait behind large frames.  Host code only; every step runs in
// the codec kernels.
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
    int inflight = 0;   // requests in steps on the device (in consecutive steps, completing in order)
};

constexpr int kMaxDepth = 8;   // steps in flight per shard, at most

// one enqueued step of a shard: its requests by slot (kind 0: none), the
// record-ring slot its results come back in, and its completion event
struct Step {
    cudaEvent_t ev = nullptr;
    int ring = 0;
    int mode = 0;
    int64_t t_launch = 0;
    std::vector<Request> req;
};

struct Shard {
    Core core;
    cvc_params prm;
    cudaStream_t st = nullptr;
    std::deque<Step> flying;          // in launch order, at most the server's depth
    std::vector<cudaEvent_t> events;  // one per step in flight, handed to steps in turn
    int next_event = 0;
    std::vector<int> slot_session;    // -1: free
    std::vector<int> slot_flying;     // requests of the slot in flight
    size_t bytes = 0;
    bool busy() const { return !flying.empty(); }
    int live() const {
        int n = 0;
        for (int s : slot_session) n += s >= 0;
        return n;
    }
    ~Shard() {
        for (cudaEvent_t e : events)
            if (e) cudaEventDestroy(e);
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
    int depth = 1;   // steps in flight per shard
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

    void complete(Shard* sh, Step& step, int slot, cvc_status fail) {
        Request& r = step.req[slot];
        cvc_server_completion cpl;
        memset(&cpl, 0, sizeof(cpl));
        cpl.tag = r.tag;
        cpl.session = sh->slot_session[slot];
        cpl.kind = r.kind;
        cpl.frame_type = cpl.dec_frame_type = -1;
        if (fail == CVC_OK) {
            unsigned didx = 0;
            core_commit_at(&sh->core, step.ring, slot, &cpl.enc_status, &cpl.dec_status, &cpl.out_len,
                           &cpl.frame_type, &cpl.dec_frame_type, &didx);
        } else {
            cpl.enc_status = (r.kind & 1) ? fail : CVC_OK;
            cpl.dec_status = (r.kind & 2) ? fail : CVC_OK;
        }
        cpl.t_submit_ns = r.t_submit;
        cpl.t_launch_ns = step.t_launch;
        cpl.t_done_ns = now_ns();
        done.push_back(cpl);
        requests_done++;
        r.kind = 0;
        sh->slot_flying[slot]--;
        sessions[cpl.session].inflight--;
    }

    // collect finished steps, oldest first per shard; returns the number of steps that finished
    int reap() {
        int n = 0;
        for (auto& up : shards) {
            Shard* sh = up.get();
            while (sh && sh->busy()) {
                Step& step = sh->flying.front();
                cudaError_t q = cudaEventQuery(step.ev);
                if (q == cudaErrorNotReady) break;
                cvc_status fail = CVC_OK;
                if (q != cudaSuccess) {
                    cudaGetLastError();
                    fail = CVC_ERR_CUDA;
                    sticky = CVC_ERR_CUDA;
                }
                for (int s = 0; s < (int)step.req.size(); s++)
                    if (step.req[s].kind) complete(sh, step, s, fail);
                sh->flying.pop_front();
                n++;
            }
        }
        return n;
    }

    void retire() {
        for (int id = 0; id < (int)sessions.size(); id++) {
            Session& S = sessions[id];
            if (S.state == S_DONE || !S.closing || !S.q.empty() || S.inflight > 0) continue;
            if (S.state == S_WAITING) {
                waiting.erase(std::remove(waiting.begin(), waiting.end(), id), waiting.end());
            } else {
                shards[S.shard]->slot_session[S.slot] = -1;
            }
            S.state = S_DONE;
        }
        for (auto& up : shards) {
            if (!up || up->busy() || up->live() > 0) continue;
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
        // smaller frames, shorter steps: a higher stream priority (numerically lower), so that
        // they do not wait behind the kernels of large frames
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            cudaGetLastError();
            least = greatest = 0;
        }
        const long long px = (long long)p.width * p.height;
        const int prio = px <= 110000 ? greatest : (px <= 400000 ? (least + greatest) / 2 : least);
        if (cudaStreamCreateWithPriority(&sh->st, cudaStreamNonBlocking, prio) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        sh->events.assign(depth, nullptr);
        for (cudaEvent_t& e : sh->events)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                e = nullptr;
                cudaGetLastError();
                return false;
            }
        sh->prm = p;
        sh->bytes = bytes;
        sh->slot_session.assign(cfg.slots_per_shard, -1);
        sh->slot_flying.assign(cfg.slots_per_shard, 0);
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
                    if (sh->slot_session[s] < 0 && !sh->slot_flying[s]) {
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
            if (!sh || (int)sh->flying.size() >= depth) continue;
            Step step;
            step.req.assign(sh->slot_session.size(), Request{0, {}, 0, 0});
            int mode = 0;
            for (int s = 0; s < (int)sh->slot_session.size(); s++) {
                const int id = sh->slot_session[s];
                if (id < 0) continue;
                Session& S = sessions[id];
                // one request per session per step; a session's later requests go into later
                // steps, which the shard's stream runs in order
                if (S.q.empty()) continue;
                step.req[s] = S.q.front();
                S.q.pop_front();
                S.inflight++;
                sh->slot_flying[s]++;
                mode |= step.req[s].kind;
            }
            if (!mode) continue;
            const StreamIo none{nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0};
            cvc_status st = core_begin(&sh->core) ? CVC_OK : CVC_ERR_CUDA;
            for (int s = 0; s < (int)sh->slot_session.size() && st == CVC_OK; s++)
                core_fill_call(&sh->core, s, mode, step.req[s].kind ? stream_io(step.req[s]) : none);
            step.mode = mode;
            step.t_launch = now_ns();
            step.ring = core_ring_slot(&sh->core);
            step.ev = sh->events[sh->next_event];
            if (st == CVC_OK) st = core_enqueue(&sh->core, mode, sh->st);
            if (st == CVC_OK && cudaEventRecord(step.ev, sh->st) != cudaSuccess) st = CVC_ERR_CUDA;
            if (st != CVC_OK) {
                cudaGetLastError();
                sticky = st;
                for (int s = 0; s < (int)step.req.size(); s++)
                    if (step.req[s].kind) complete(sh, step, s, st);
                continue;
            }
            sh->next_event = (sh->next_event + 1) % depth;
            sh->flying.push_back(std::move(step));
            steps++;
        }
    }

    bool any_busy() const {
        for (auto& up : shards)
            if (up && up->busy()) return true;
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
    if (!cfg || cfg->slots_per_shard < 1 || cfg->slots_per_shard > 256 || cfg->budget_bytes == 0 ||
        cfg->steps_in_flight < 0 || cfg->steps_in_flight > kMaxDepth)
        return CVC_ERR_INVALID_ARG;
    cvc_server* s = new (std::nothrow) cvc_server();
    if (!s) return CVC_ERR_NOMEM;
    s->cfg = *cfg;
    s->depth = cfg->steps_in_flight > 0 ? cfg->steps_in_flight : 1;
    *out = s;
    return CVC_OK;
}

cvc_status cvc_server_destroy(cvc_server* s) {
    if (!s) return CVC_OK;
    for (auto& up : s->shards)
        if (up)
            for (Step& step : up->flying) cudaEventSynchronize(step.ev);
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
