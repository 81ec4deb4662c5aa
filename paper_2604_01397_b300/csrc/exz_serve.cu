// exz_serve.cu -- continuous-batching request server for the correction.
//
// A server owns one device arena sized from an HBM budget.  A host thread runs
// the pass loop of Algorithm 1 over every resident field at once and, at each
// pass boundary,
//   - admits queued requests (first come, first served) while a field slot and
//     arena room are free: the request's f and f_hat are copied in on a copy
//     stream, and its set-up (descriptor of f, first checks, CP compaction and
//     sort, first CP-pair check) joins the next pass on the compute stream;
//   - runs one pass (check, CP pairs, apply, bookkeeping) covering all
//     resident fields, whatever their sizes;
//   - retires fields that reached their fixpoint: residual check, status and
//     edit list on the compute stream, then the results go out on the copy
//     stream and a host function on that stream frees the arena room.
// A field's passes are exactly those it runs alone (fields never interact), so
// every result equals exactz_correct's for the same input.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "exactz.h"
#include "exz_common.cuh"
#include "exz_launch.h"

using namespace exz;

namespace {

using Clock = std::chrono::steady_clock;
double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }
uint64_t rup(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// First-fit allocator of aligned ranges of [0, cap).
class Arena {
  public:
    void init(uint64_t cap)
    {
        free_.clear();
        if (cap) free_[0] = cap;
    }
    bool alloc(uint64_t len, uint64_t align, uint64_t &off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const uint64_t a = rup(it->first, align), end = it->first + it->second;
            if (a + len > end) continue;
            const uint64_t s0 = it->first, s1 = a + len;
            free_.erase(it);
            if (a > s0) free_[s0] = a - s0;
            if (end > s1) free_[s1] = end - s1;
            off = a;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t len)
    {
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<uint64_t, uint64_t> free_;  // offset -> length
};

enum { Q_QUEUED = 0, Q_RESIDENT = 1, Q_COPYING = 2, Q_DONE = 3 };

struct Req {
    exactz_server *S = nullptr;
    uint64_t ticket = 0;
    const float *f = nullptr, *fhat = nullptr;
    float xi = 0.f;
    float *g_out = nullptr;
    exactz_edit *edits_out = nullptr;
    FieldDesc fd{};  // geometry; arena offsets are added at admission
    // sizes in the five arenas (vertices, row words, tiles, CP entries, edits) and their offsets
    uint64_t n = 0, nv = 0, nw = 0, nt = 0, ne = 0;
    uint64_t v0 = 0, w0 = 0, t0 = 0, c0 = 0, e0 = 0;
    uint32_t slot = 0;
    int state = Q_QUEUED;
    double t_submit = 0, t_done = 0;
    exactz_result res{};
};

}  // namespace

struct exactz_server {
    int device = 0;
    uint32_t slots = 0;
    exactz_opts opts{};
    uint64_t V = 0, W = 0, T = 0, C = 0, E = 0;  // arena capacities
    uint64_t bytes = 0;
    std::vector<void *> allocs;

    FieldDesc *d_fields = nullptr;
    FieldState *d_fst = nullptr;
    LoopState *d_ls = nullptr;
    uint32_t *d_multi = nullptr;
    float *f = nullptr, *fhat = nullptr, *g = nullptr;
    uint32_t *desc = nullptr, *cp_rank = nullptr;
    uint32_t *cpwords = nullptr, *reqw = nullptr, *dirty = nullptr;
    uint8_t *tile_flag = nullptr, *apply_flag = nullptr;
    uint32_t *pin_tile_bits = nullptr, *pin_tile_arena = nullptr, *tile_field = nullptr;
    uint32_t *cp_key[2] = {nullptr, nullptr};
    unsigned long long *cp_ent[2] = {nullptr, nullptr};
    float *gs = nullptr;
    uint32_t *pairbits = nullptr, *pin_pair_arena = nullptr;
    EditRec *edits = nullptr;
    uint32_t *blk = nullptr;
    unsigned long long *blk_off = nullptr;
    uint32_t *hist = nullptr;
    uint32_t sort_blocks = 0;
    uint32_t *d_retire = nullptr;
    CUtensorMap *d_tmaps = nullptr;  // TMA maps of each slot's f, f_hat, g, descriptors (TMAPS per slot)

    FieldState *h_fst = nullptr;
    FieldDesc *h_fd = nullptr;
    CUtensorMap *h_tmaps = nullptr;
    uint32_t *h_retire = nullptr;
    cudaStream_t cs = nullptr, xs = nullptr;  // compute, copy
    cudaEvent_t in_ev = nullptr;               // inputs landed (re-recorded per admission)
    cudaEvent_t refl_ev = nullptr;             // increasing edits: the room's g is free for the next input

    // guarded by mu
    Arena av, aw, at, ac, ae;
    std::vector<uint32_t> free_slots;
    std::deque<Req *> queue;
    std::vector<Req *> running;
    uint64_t copying = 0;
    std::unordered_map<uint64_t, Req *> reqs;
    bool stop = false;
    int error = 0;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, cancelled = 0, passes = 0, max_resident = 0, admitted_vertices = 0;
    std::atomic<uint64_t> launches{0};  // written by the serving thread
    double busy_s = 0;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::thread th;
};

namespace {

void free_server(exactz_server *S)
{
    if (S->xs) cudaStreamSynchronize(S->xs);  // pending completion callbacks touch S
    if (S->cs) cudaStreamSynchronize(S->cs);
    cudaGetLastError();
    if (S->cs) cudaStreamDestroy(S->cs);
    if (S->xs) cudaStreamDestroy(S->xs);
    if (S->in_ev) cudaEventDestroy(S->in_ev);
    if (S->refl_ev) cudaEventDestroy(S->refl_ev);
    for (void *p : S->allocs) cudaFree(p);
    if (S->h_fst) cudaFreeHost(S->h_fst);
    if (S->h_fd) cudaFreeHost(S->h_fd);
    if (S->h_tmaps) cudaFreeHost(S->h_tmaps);
    if (S->h_retire) cudaFreeHost(S->h_retire);
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
}

template <class T>
bool salloc(exactz_server *S, T *&p, uint64_t count)
{
    void *q = nullptr;
    const uint64_t bytes = std::max<uint64_t>(count, 1) * sizeof(T);
    if (dev_malloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    S->allocs.push_back(q);
    S->bytes += bytes;
    p = static_cast<T *>(q);
    return true;
}

Dev server_dev(const exactz_server *S)
{
    Dev D{};
    D.fields = S->d_fields;
    D.fst = S->d_fst;
    D.ls = S->d_ls;
    D.nfields = S->slots;
    D.total_tiles = (uint32_t)S->T;
    D.total_v = S->V;
    D.total_w = S->W;
    D.desc = S->desc;
    D.cp_rank = S->cp_rank;
    D.cpwords = S->cpwords;
    D.reqw = S->reqw;
    D.dirty = S->dirty;
    D.gs = S->gs;
    D.pairbits = S->pairbits;
    D.apply_flag = S->apply_flag;
    D.tile_flag = S->tile_flag;
    D.pin_tile_bits = S->pin_tile_bits;
    D.cp_key[0] = S->cp_key[0];
    D.cp_key[1] = S->cp_key[1];
    D.cp_ent[0] = S->cp_ent[0];
    D.cp_ent[1] = S->cp_ent[1];
    D.o = S->cp_ent[sort_passes(0, 1) & 1];  // every set-up sorts one field
    D.multi = S->d_multi;
    D.cp_cap = S->C;
    D.blk = S->blk;
    D.blk_off = S->blk_off;
    D.hist = S->hist;
    D.sort_blocks = S->sort_blocks;
    D.tile_field = S->tile_field;
    D.tmaps = S->d_tmaps;
    D.tun = Tuning{};  // default launch schedule
    return D;
}

// Geometry of one field (tiles, row words), independent of where it is placed.
bool geometry(const exactz_dims &d, FieldDesc &F, uint64_t &nw, uint64_t &nt)
{
    const uint64_t nx = d.nx, ny = d.ny, nz = d.nz;
    if (nx < 1 || ny < 1 || nz < 1) return false;
    const uint64_t n = nx * ny * nz;
    if (n < 2) return false;
    std::memset(&F, 0, sizeof(F));
    F.nx = (uint32_t)nx;
    F.ny = (uint32_t)ny;
    F.nz = (uint32_t)nz;
    F.n = n;
    F.tnx = (uint32_t)((nx + TX - 1) / TX);
    F.tny = (uint32_t)((ny + TY - 1) / TY);
    F.tnz = (uint32_t)((nz + TZ - 1) / TZ);
    F.div_nx = make_fastdiv(F.nx);
    F.div_ny = make_fastdiv(F.ny);
    F.div_tnx = make_fastdiv(F.tnx);
    F.div_tny = make_fastdiv(F.tny);
    nw = ny * nz * F.tnx;
    nt = (uint64_t)F.tnx * F.tny * F.tnz;
    return true;
}

// Reserve a slot and arena room for r; false leaves everything as it was.
// Vertex and word ranges start on the blocks of the compaction kernels, tile
// and CP ranges on 32-entry bitmap words, so no bitmap word is shared.
bool try_reserve(exactz_server *S, Req *r)
{
    if (S->free_slots.empty()) return false;
    uint64_t v0, w0 = 0, t0 = 0, c0 = 0, e0 = 0;
    if (!S->av.alloc(r->nv, VBLOCK, v0)) return false;
    bool ok = S->aw.alloc(r->nw, WBLOCK, w0);
    if (ok && !(ok = S->at.alloc(r->nt, 32, t0))) S->aw.release(w0, r->nw);
    if (ok && !(ok = S->ac.alloc(r->n, 32, c0))) {
        S->aw.release(w0, r->nw);
        S->at.release(t0, r->nt);
    }
    if (ok && r->ne && !(ok = S->ae.alloc(r->ne, 1, e0))) {
        S->aw.release(w0, r->nw);
        S->at.release(t0, r->nt);
        S->ac.release(c0, r->n);
    }
    if (!ok) {
        S->av.release(v0, r->nv);
        return false;
    }
    r->v0 = v0;
    r->w0 = w0;
    r->t0 = t0;
    r->c0 = c0;
    r->e0 = e0;
    r->slot = S->free_slots.back();
    S->free_slots.pop_back();
    return true;
}

void release_room(exactz_server *S, Req *r)
{
    S->av.release(r->v0, r->nv);
    S->aw.release(r->w0, r->nw);
    S->at.release(r->t0, r->nt);
    S->ac.release(r->c0, r->n);
    if (r->ne) S->ae.release(r->e0, r->ne);
    S->free_slots.push_back(r->slot);
}

// Runs on the copy stream once a request's results are in host memory.  It
// makes no CUDA call: it records the time, frees the room and wakes waiters.
void CUDART_CB on_copied(void *p)
{
    Req *r = static_cast<Req *>(p);
    exactz_server *S = r->S;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->t_done = now_s();
        r->state = Q_DONE;
        release_room(S, r);
        S->copying--;
        S->completed++;
    }
    S->done_cv.notify_all();
    S->cv.notify_all();
}

#define SK(x)                     \
    do {                          \
        if ((x) != cudaSuccess) { \
            cudaGetLastError();   \
            return EXACTZ_ENODEV; \
        }                         \
    } while (0)

// Copy the request in, clear its room, and launch its set-up and first checks.
int start_request(exactz_server *S, const Dev &D, Req *r)
{
    const uint32_t slot = r->slot;
    FieldDesc F = r->fd;
    F.N = S->opts.N;
    F.xi = r->xi;
    F.delta = r->xi / (float)S->opts.N;  // binary32 division, Sec. 3.3
    F.max_iters = S->opts.max_iters;
    F.tbase = r->t0;
    F.vbase = r->v0;
    F.wbase = r->w0;
    F.f = S->f + r->v0;
    F.fhat = S->fhat + r->v0;
    F.g = S->g + r->v0;
    F.edits = r->ne ? S->edits + r->e0 : nullptr;
    F.edits_cap = r->ne;
    F.pin_tiles = S->pin_tile_arena + r->t0;
    F.pin_pairs = S->pin_pair_arena + 2 * r->c0;
    const bool inc = S->opts.direction == EXACTZ_EDITS_INCREASING;
    F.mirror = inc ? 1u : 0u;  // increasing edits: the room holds the reflection of -f, -f_hat
    // tile loads by TMA where the room's arrays can be mapped (else cp.async)
    CUtensorMap *m = S->h_tmaps + (uint64_t)TMAPS * slot;
    F.tma = (make_map(m, F.f, F, true) && make_map(m + 1, F.fhat, F, true) ? TMA_SETUP : 0u) |
            (make_map(m + 2, F.g, F, true) ? TMA_G : 0u) | (make_map(m + 3, S->desc + r->v0, F, false) ? TMA_DESC : 0u);
    S->h_fd[slot] = F;
    if (!inc) {
        SK(cudaMemcpyAsync(S->f + r->v0, r->f, r->n * 4, cudaMemcpyHostToDevice, S->xs));
        SK(cudaMemcpyAsync(S->fhat + r->v0, r->fhat, r->n * 4, cudaMemcpyHostToDevice, S->xs));
    } else {
        // each input lands in the room's g (free until the set-up) and is
        // reflected from there into f or f_hat, v -> n-1-v with negation
        float *stage = S->g + r->v0;
        SK(cudaMemcpyAsync(stage, r->f, r->n * 4, cudaMemcpyHostToDevice, S->xs));
        SK(cudaEventRecord(S->in_ev, S->xs));
        SK(cudaStreamWaitEvent(S->cs, S->in_ev, 0));
        launch_reflect_in(stage, S->f + r->v0, r->n, S->cs);
        SK(cudaEventRecord(S->refl_ev, S->cs));
        SK(cudaStreamWaitEvent(S->xs, S->refl_ev, 0));
        SK(cudaMemcpyAsync(stage, r->fhat, r->n * 4, cudaMemcpyHostToDevice, S->xs));
        SK(cudaEventRecord(S->in_ev, S->xs));
        SK(cudaStreamWaitEvent(S->cs, S->in_ev, 0));
        launch_reflect_in(stage, S->fhat + r->v0, r->n, S->cs);
        S->launches += 2;
    }
    SK(cudaEventRecord(S->in_ev, S->xs));
    // meanwhile clear the room on the compute stream (it may hold an earlier field's state)
    SK(cudaMemcpyAsync(S->d_fields + slot, &S->h_fd[slot], sizeof(FieldDesc), cudaMemcpyHostToDevice, S->cs));
    if (F.tma)
        SK(cudaMemcpyAsync(S->d_tmaps + (uint64_t)TMAPS * slot, m, sizeof(CUtensorMap) * TMAPS, cudaMemcpyHostToDevice,
                           S->cs));
    SK(cudaMemsetAsync(S->d_fst + slot, 0, sizeof(FieldState), S->cs));
    SK(cudaMemsetAsync(S->desc + r->v0, 0, r->nv * 4, S->cs));
    SK(cudaMemsetAsync(S->cpwords + r->w0, 0, r->nw * 4, S->cs));
    SK(cudaMemsetAsync(S->reqw + r->w0, 0, r->nw * 4, S->cs));
    SK(cudaMemsetAsync(S->dirty + r->w0, 0, r->nw * 4, S->cs));
    const uint64_t tw0 = r->t0 / 32, tw1 = (r->t0 + r->nt + 31) / 32;
    SK(cudaMemsetAsync(S->pin_tile_bits + tw0, 0, (tw1 - tw0) * 4, S->cs));
    SK(cudaMemsetAsync(S->tile_flag + r->t0, 0, r->nt, S->cs));
    SK(cudaMemsetAsync(S->apply_flag + r->t0, 0, r->nt, S->cs));
    const uint64_t cw0 = r->c0 / 32, cw1 = (r->c0 + r->n + 31) / 32;
    SK(cudaMemsetAsync(S->pairbits + cw0, 0, (cw1 - cw0) * 4, S->cs));
    launch_fill_u32(S->tile_field + r->t0, slot, r->nt, S->cs);
    SK(cudaStreamWaitEvent(S->cs, S->in_ev, 0));
    const SetupRange R{(uint32_t)r->t0, (uint32_t)(r->t0 + r->nt), r->w0 / WBLOCK, r->nw / WBLOCK,
                       slot, slot + 1, r->c0, &S->d_fst[slot].ncp};
    launch_setup(D, R, S->cs);
    launch_cp_compact(D, R, S->cs);
    launch_cp_sort(D, R, S->cs);
    launch_pairs_all(D, R, S->cs);
    S->launches += 1 + 1 + 4 + 3 * sort_passes(slot, slot + 1) + 1;  // fill, setup, compaction, sort, pairs
    SK(cudaGetLastError());
    return EXACTZ_OK;
}

// Residual check, status and edit list of the finished fields; copy results out.
int retire(exactz_server *S, const Dev &D, const std::vector<Req *> &fin)
{
    const uint32_t nf = (uint32_t)fin.size();
    for (uint32_t i = 0; i < nf; i++) S->h_retire[i] = fin[i]->slot;
    SK(cudaMemcpyAsync(S->d_retire, S->h_retire, 4ull * nf, cudaMemcpyHostToDevice, S->cs));
    const FieldSet FS{S->d_retire, nf, 0, 0, 0, 0};
    launch_check_pinned(D, FS, S->cs);
    launch_pairs_pinned(D, FS, S->cs);
    launch_finish(D, FS, S->cs);
    for (uint32_t i = 0; i < nf; i++) {
        const Req *r = fin[i];
        const FieldSet one{S->d_retire + i, 1, r->v0 / VBLOCK, r->nv / VBLOCK, r->slot, r->slot + 1};
        launch_edit_list(D, one, r->ne ? 1 : 0, S->cs);
        S->launches += r->ne ? 3 : 1;
        if (S->opts.direction == EXACTZ_EDITS_INCREASING) {  // g back in the caller's coordinates and sign
            launch_reflect_out(S->g + r->v0, S->desc + r->v0, r->n, S->cs);
            S->launches += 1;
        }
    }
    S->launches += 4;  // pinned checks, pinned pairs, residual count, status
    SK(cudaGetLastError());
    SK(cudaMemcpyAsync(S->h_fst, S->d_fst, sizeof(FieldState) * S->slots, cudaMemcpyDeviceToHost, S->cs));
    SK(cudaStreamSynchronize(S->cs));
    for (Req *r : fin) {
        const FieldState &st = S->h_fst[r->slot];
        exactz_result &R = r->res;
        std::memset(&R, 0, sizeof(R));
        R.iterations = st.iterations;
        R.n_edits = st.n_edits;
        R.n_lossless = st.n_lossless;
        R.residual_violations = st.capped + st.pinned_res;
        R.n_critical = st.ncp;
        R.status = (int32_t)st.status;
        SK(cudaMemcpyAsync(r->g_out, S->g + r->v0, r->n * 4, cudaMemcpyDeviceToHost, S->xs));
        const uint64_t ne = std::min<uint64_t>(st.n_edits, r->ne);
        if (ne)
            SK(cudaMemcpyAsync(r->edits_out, S->edits + r->e0, ne * sizeof(EditRec), cudaMemcpyDeviceToHost, S->xs));
        SK(cudaLaunchHostFunc(S->xs, on_copied, r));
    }
    return EXACTZ_OK;
}

void serve(exactz_server *S)
{
    cudaSetDevice(S->device);
    const Dev D = server_dev(S);
    std::vector<Req *> admit, fin;
    for (;;) {
        admit.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] {
                return (S->stop && S->queue.empty()) || !S->running.empty() ||
                       (!S->queue.empty() && !S->free_slots.empty());
            });
            if (S->stop && S->queue.empty() && S->running.empty()) break;
            while (!S->queue.empty()) {
                Req *r = S->queue.front();
                if (!try_reserve(S, r)) break;
                S->queue.pop_front();
                r->state = Q_RESIDENT;
                S->admitted_vertices += r->n;
                admit.push_back(r);
                S->running.push_back(r);
            }
            if (S->running.empty()) {
                // nothing resident and the head does not fit: the room it needs
                // is held by results still being copied out
                S->cv.wait(lk, [&] { return S->copying == 0; });
                continue;
            }
        }
        const double t0 = now_s();
        int rc = EXACTZ_OK;
        for (Req *r : admit)
            if (!rc) rc = start_request(S, D, r);
        fin.clear();
        if (!rc) {
            launch_check_list(D, S->cs);
            launch_pairs_list(D, S->cs);
            launch_apply(D, 1, S->cs);
            launch_book(D, 0, 0, S->cs);
            S->launches += 4;
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(S->h_fst, S->d_fst, sizeof(FieldState) * S->slots, cudaMemcpyDeviceToHost,
                                S->cs) != cudaSuccess ||
                cudaStreamSynchronize(S->cs) != cudaSuccess)
                rc = EXACTZ_ENODEV;
        }
        if (!rc) {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Req *r : S->running)
                if (S->h_fst[r->slot].done) fin.push_back(r);
            for (Req *r : fin) {
                S->running.erase(std::find(S->running.begin(), S->running.end(), r));
                r->state = Q_COPYING;
                S->copying++;
            }
        }
        if (!rc && !fin.empty()) rc = retire(S, D, fin);
        std::lock_guard<std::mutex> lk(S->mu);
        S->passes++;
        S->busy_s += now_s() - t0;
        S->max_resident = std::max<uint64_t>(S->max_resident, S->running.size() + fin.size());
        if (rc) {
            S->error = rc;  // a CUDA failure ends the server; waiters see the error
            S->stop = true;
            S->done_cv.notify_all();
            break;
        }
    }
}

}  // namespace

extern "C" {

exactz_server *exactz_server_create(const exactz_server_config *cfg)
{
    if (!cfg || cfg->budget_bytes < (64ull << 20) || cfg->max_fields < 1 || cfg->max_fields > 4096) return nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return nullptr;
    }
    exactz_opts o;
    exactz_default_opts(&o);
    if (cfg->opts.N) o = cfg->opts;
    if (o.N < 1 || o.N > 254 || o.events != EXACTZ_EVENTS_REFORMULATED || o.direction > EXACTZ_EDITS_INCREASING)
        return nullptr;
    exactz_server *S = new (std::nothrow) exactz_server();
    if (!S) return nullptr;
    cudaGetDevice(&S->device);
    S->slots = cfg->max_fields;
    S->opts = o;
    // Arena capacities from the budget: 1/8 for edit records, the rest at
    // 60 bytes per resident vertex (f, f_hat, g, descriptor, CP rank: 20; one
    // CP slot per vertex for keys, entries, sorted values, pinned pairs: 36;
    // row words, tiles and rounding: the rest).
    const uint64_t B = cfg->budget_bytes;
    S->E = B / 8 / sizeof(EditRec);
    S->V = (B - S->E * sizeof(EditRec)) / 60 / VBLOCK * VBLOCK;
    S->C = S->V;
    S->W = rup(S->V / 16 + (uint64_t)S->slots * WBLOCK, WBLOCK);
    S->T = rup(S->V / 256 + (uint64_t)S->slots * 32, 32);
    S->sort_blocks = (uint32_t)device_sms() * 2;
    const uint64_t V = S->V, W = S->W, T = S->T, C = S->C;
    const uint64_t nblk = std::max(V / VBLOCK, W / WBLOCK) + 1;
    bool ok = salloc(S, S->d_fields, S->slots) && salloc(S, S->d_fst, S->slots) && salloc(S, S->d_ls, 1) &&
              salloc(S, S->d_multi, 512) && salloc(S, S->f, V) && salloc(S, S->fhat, V) && salloc(S, S->g, V) &&
              salloc(S, S->desc, V) && salloc(S, S->cp_rank, V) && salloc(S, S->cpwords, W) &&
              salloc(S, S->reqw, W) && salloc(S, S->dirty, W) && salloc(S, S->tile_flag, T) &&
              salloc(S, S->apply_flag, T) &&
              salloc(S, S->pin_tile_bits, T / 32 + 1) && salloc(S, S->pin_tile_arena, T) &&
              salloc(S, S->tile_field, T) && salloc(S, S->cp_key[0], C) && salloc(S, S->cp_key[1], C) &&
              salloc(S, S->cp_ent[0], C) && salloc(S, S->cp_ent[1], C) && salloc(S, S->gs, C) &&
              salloc(S, S->pairbits, C / 32 + 1) && salloc(S, S->pin_pair_arena, 2 * C) &&
              salloc(S, S->edits, S->E) && salloc(S, S->blk, nblk) && salloc(S, S->blk_off, nblk) &&
              salloc(S, S->hist, 256ull * S->sort_blocks) && salloc(S, S->d_retire, S->slots) &&
              salloc(S, S->d_tmaps, (uint64_t)TMAPS * S->slots);
    ok = ok && cudaMallocHost(&S->h_fst, sizeof(FieldState) * S->slots) == cudaSuccess &&
         cudaMallocHost(&S->h_fd, sizeof(FieldDesc) * S->slots) == cudaSuccess &&
         cudaMallocHost(&S->h_tmaps, sizeof(CUtensorMap) * TMAPS * S->slots) == cudaSuccess &&
         cudaMallocHost(&S->h_retire, 4ull * S->slots) == cudaSuccess &&
         cudaStreamCreateWithFlags(&S->cs, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&S->xs, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&S->in_ev, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&S->refl_ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        // every slot starts out finished; the loop state and the bitmaps start clear
        std::vector<FieldState> idle(S->slots);
        std::memset(idle.data(), 0, sizeof(FieldState) * S->slots);
        for (auto &st : idle) st.done = 1;
        ok = cudaMemcpy(S->d_fst, idle.data(), sizeof(FieldState) * S->slots, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(S->d_ls, 0, sizeof(LoopState)) == cudaSuccess &&
             cudaMemcpy(S->d_multi, host_multi_table(), 2048, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(S->reqw, 0, W * 4) == cudaSuccess && cudaMemset(S->dirty, 0, W * 4) == cudaSuccess &&
             cudaMemset(S->tile_flag, 0, T) == cudaSuccess && cudaMemset(S->apply_flag, 0, T) == cudaSuccess &&
             cudaMemset(S->pin_tile_bits, 0, (T / 32 + 1) * 4) == cudaSuccess &&
             cudaMemset(S->pairbits, 0, (C / 32 + 1) * 4) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_server(S);
        return nullptr;
    }
    S->av.init(V);
    S->aw.init(W);
    S->at.init(T);
    S->ac.init(C);
    S->ae.init(S->E);
    for (uint32_t i = 0; i < S->slots; i++) S->free_slots.push_back(S->slots - 1 - i);
    S->th = std::thread(serve, S);
    return S;
}

int exactz_server_submit(exactz_server *S, const float *f, const float *fhat, exactz_dims d, float xi,
                         float *g_out, exactz_edit *edits_out, uint64_t edits_cap, uint64_t *ticket)
{
    if (!S || !f || !fhat || !g_out || !ticket || !(xi > 0.0f) || !std::isfinite(xi)) return EXACTZ_EINVAL;
    Req *r = new (std::nothrow) Req();
    if (!r) return EXACTZ_ENOMEM;
    uint64_t nw = 0, nt = 0;
    if (!geometry(d, r->fd, nw, nt)) {
        delete r;
        return EXACTZ_EINVAL;
    }
    r->S = S;
    r->f = f;
    r->fhat = fhat;
    r->xi = xi;
    r->g_out = g_out;
    r->edits_out = edits_out;
    r->n = r->fd.n;
    r->nv = rup(r->n, VBLOCK);
    r->nw = rup(nw, WBLOCK);
    r->nt = nt;
    r->ne = (edits_out && S->opts.want_edit_list) ? std::min<uint64_t>(edits_cap, r->n) : 0;
    if (r->n >= (1ull << 32) || r->nv > S->V || r->nw > S->W || r->nt > S->T || r->n > S->C || r->ne > S->E) {
        delete r;
        return EXACTZ_ESIZE;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return S->error ? S->error : EXACTZ_EINVAL;
        }
        r->ticket = S->next_ticket++;
        r->t_submit = now_s();
        S->reqs[r->ticket] = r;
        S->queue.push_back(r);
        S->submitted++;
        *ticket = r->ticket;
    }
    S->cv.notify_all();
    return EXACTZ_OK;
}

static int take_result(exactz_server *S, Req *r, exactz_result *res, double *latency_s)
{
    if (res) *res = r->res;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    S->reqs.erase(r->ticket);
    delete r;
    return 1;
}

int exactz_server_poll(exactz_server *S, uint64_t ticket, exactz_result *res, double *latency_s)
{
    if (!S) return EXACTZ_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return EXACTZ_EINVAL;
    if (it->second->state == Q_DONE) return take_result(S, it->second, res, latency_s);
    return S->error ? S->error : 0;
}

int exactz_server_wait(exactz_server *S, uint64_t ticket, double timeout_s, exactz_result *res, double *latency_s)
{
    if (!S) return EXACTZ_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return EXACTZ_EINVAL;
    Req *r = it->second;
    const double lim = (timeout_s < 0 || timeout_s > 1e6) ? 1e6 : timeout_s;
    const auto deadline =
        Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(lim));
    S->done_cv.wait_until(lk, deadline, [&] { return r->state == Q_DONE || S->error != 0; });
    if (r->state == Q_DONE) return take_result(S, r, res, latency_s);
    return S->error ? S->error : 0;
}

int exactz_server_cancel(exactz_server *S, uint64_t ticket)
{
    if (!S) return EXACTZ_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return EXACTZ_EINVAL;
    Req *r = it->second;
    if (r->state != Q_QUEUED) return 0;  // admitted or finished: its result comes as usual
    auto q = std::find(S->queue.begin(), S->queue.end(), r);
    if (q != S->queue.end()) S->queue.erase(q);
    S->reqs.erase(it);
    S->cancelled++;
    delete r;
    return 1;
}

int exactz_server_stats(exactz_server *S, exactz_server_info *out)
{
    if (!S || !out) return EXACTZ_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->passes = S->passes;
    out->max_resident = S->max_resident;
    out->resident = S->running.size();
    out->queued = S->queue.size();
    out->admitted_vertices = S->admitted_vertices;
    out->capacity_vertices = S->V;
    out->device_bytes = S->bytes;
    out->kernel_launches = S->launches.load();
    out->busy_s = S->busy_s;
    out->error = S->error;
    out->cancelled = S->cancelled;
    return EXACTZ_OK;
}

void exactz_server_destroy(exactz_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    free_server(S);
}

}  // extern "C"
