// exz_engine.cu -- host side of the B300 EXaCTz correction: workspace layout,
// the iterate-to-fixpoint loop of Algorithm 1 in three forms, and the C ABI.
//
// One run over F fields (F = 1 for exactz_correct):
//   set-up     k_stencil<SETUP> (descriptor of f, g := f_hat, first checks),
//              ordered CP compaction, stable radix sort by (field, value),
//              reformulated event check on all CP pairs, apply, bookkeeping;
//   loop       PLAIN:    full sweep + all pairs each pass, host reads the flag;
//              FRONTIER: only tiles / pairs touched by the last pass's edits;
//              GRAPH:    the FRONTIER pass as the body of a CUDA-graph
//                        conditional while-node; the bookkeeping kernel clears
//                        the condition when every field is done;
//   finish     pinned-vertex residual check, status, edit-list compaction.
// All three forms compute identical results (the frontier only skips checks
// whose requests would target pinned vertices; see the oracle's notes).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include <cudaTypedefs.h>

#include "exactz.h"
#include "exz_common.cuh"
#include "exz_launch.h"

using namespace exz;

namespace {

uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------- link table
// multi[S] = 1 iff the link subgraph induced on the neighbour subset S (bit s =
// rank rank_of(s)) has at least two connected components.  Two neighbours are
// linked iff their offsets differ by a neighbour offset.
uint32_t g_multi_host[512];
std::once_flag g_multi_once;

void build_multi_table()
{
    uint32_t adj[14] = {0};
    for (int a = 0; a < 14; a++)
        for (int b = 0; b < 14; b++) {
            if (a == b) continue;
            const int ra = rank_of(a), rb = rank_of(b);
            const int dx = rdx(rb) - rdx(ra), dy = rdy(rb) - rdy(ra), dz = rdz(rb) - rdz(ra);
            const bool pos = dx >= 0 && dy >= 0 && dz >= 0, neg = dx <= 0 && dy <= 0 && dz <= 0;
            const bool nonzero = dx || dy || dz;
            const bool small = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
            if (nonzero && small && (pos || neg)) adj[a] |= 1u << b;
        }
    std::memset(g_multi_host, 0, sizeof(g_multi_host));
    for (uint32_t S = 0; S < (1u << 14); S++) {
        uint32_t rem = S;
        int comps = 0;
        while (rem) {
            uint32_t comp = rem & (~rem + 1);
            for (;;) {
                uint32_t grow = comp;
                for (int s = 0; s < 14; s++)
                    if (comp & (1u << s)) grow |= adj[s] & S;
                if (grow == comp) break;
                comp = grow;
            }
            rem &= ~comp;
            comps++;
        }
        if (comps >= 2) g_multi_host[S >> 5] |= 1u << (S & 31);
    }
}

// ---------------------------------------------------------------- layout
struct Layout {
    uint32_t nfields = 0;
    uint64_t total_v = 0, total_w = 0, total_real = 0;
    uint32_t total_tiles = 0;
    std::vector<FieldDesc> fd;
    std::vector<uint64_t> cpc;  // per field: sum of the vertex counts before it (CP capacity offset)
    // fields whose rows are not a multiple of 16 bytes: the offset and row
    // pitch of their padded copy of g (pitch 0: none)
    std::vector<uint64_t> moff;
    std::vector<uint32_t> mpitch;
    uint64_t total_mirror = 0;
};

int make_layout(uint32_t nf, const exactz_dims *d, Layout &L)
{
    if (nf == 0 || nf >= (1u << 24) || !d) return EXACTZ_EINVAL;
    L.nfields = nf;
    L.fd.assign(nf, FieldDesc{});
    L.cpc.assign(nf, 0);
    L.moff.assign(nf, 0);
    L.mpitch.assign(nf, 0);
    uint64_t v = 0, w = 0, t = 0, real = 0;
    for (uint32_t i = 0; i < nf; i++) {
        const uint64_t nx = d[i].nx, ny = d[i].ny, nz = d[i].nz;
        if (nx < 1 || ny < 1 || nz < 1) return EXACTZ_EINVAL;
        const uint64_t n = nx * ny * nz;
        if (n < 2 || n >= (1ull << LOCAL_BITS)) return EXACTZ_EINVAL;
        FieldDesc &F = L.fd[i];
        F.nx = (uint32_t)nx;
        F.ny = (uint32_t)ny;
        F.nz = (uint32_t)nz;
        F.n = n;
        F.tnx = (uint32_t)((nx + TX - 1) / TX);
        F.tny = (uint32_t)((ny + TY - 1) / TY);
        F.tnz = (uint32_t)((nz + TZ - 1) / TZ);
        F.tbase = t;
        F.div_nx = make_fastdiv(F.nx);
        F.div_ny = make_fastdiv(F.ny);
        F.div_tnx = make_fastdiv(F.tnx);
        F.div_tny = make_fastdiv(F.tny);
        t += (uint64_t)F.tnx * F.tny * F.tnz;
        v = round_up(v, VBLOCK);
        F.vbase = v;
        v += n;
        w = round_up(w, WBLOCK);
        F.wbase = w;
        w += ny * nz * F.tnx;
        L.cpc[i] = real;
        real += n;
        if (nx % 4 != 0) {
            L.mpitch[i] = (uint32_t)round_up(nx, 4);
            L.moff[i] = L.total_mirror;
            L.total_mirror = round_up(L.total_mirror + (uint64_t)L.mpitch[i] * ny * nz, 64);
        }
    }
    if (t >= (1ull << 32) || real >= (1ull << 32)) return EXACTZ_EINVAL;
    L.total_v = round_up(v, VBLOCK);
    L.total_w = round_up(w, WBLOCK);
    L.total_tiles = (uint32_t)t;
    L.total_real = real;
    return EXACTZ_OK;
}

// Key of a layout (the fields' dims in order).  A workspace remembers the key
// of its last run: padding words and vertices are cleared only when it changes.
uint64_t layout_key(uint32_t nf, const exactz_dims *d)
{
    uint64_t h = 1469598103934665603ull ^ nf;
    for (uint32_t i = 0; i < nf; i++) {
        const uint64_t v[3] = {d[i].nx, d[i].ny, d[i].nz};
        for (uint64_t x : v) h = (h ^ x) * 1099511628211ull;
    }
    return h;
}

}  // namespace

// ---------------------------------------------------------------- workspace
struct exactz_workspace {
    int device = 0;
    uint32_t cap_nf = 0;
    uint64_t cap_v = 0, cap_w = 0, cap_real = 0;
    uint32_t cap_tiles = 0;
    uint64_t bytes = 0;
    std::vector<void *> allocs;

    FieldDesc *d_fields = nullptr;
    FieldState *d_fst = nullptr;
    LoopState *d_ls = nullptr;
    uint32_t *d_multi = nullptr;
    uint32_t *desc = nullptr, *cp_rank = nullptr, *cpwords = nullptr, *reqw = nullptr;
    uint32_t *dirty = nullptr, *pairbits = nullptr;
    uint8_t *apply_flag = nullptr, *tile_flag = nullptr;
    float *gs = nullptr;
    uint32_t *pin_tile_arena = nullptr, *pin_tile_bits = nullptr;
    uint32_t *pin_pair_arena = nullptr;
    uint32_t *fids = nullptr;  // 0, 1, ..., cap_nf - 1: the set of all fields
    uint32_t *tile_field = nullptr;  // field of each tile (workspaces for several fields)
    CUtensorMap *d_tmaps = nullptr;  // TMA maps of each field's f, f_hat, g, descriptors (TMAPS per field slot)
    uint32_t *cp_key[2] = {nullptr, nullptr};
    unsigned long long *cp_ent[2] = {nullptr, nullptr};
    uint32_t *blk = nullptr;
    unsigned long long *blk_off = nullptr;
    uint32_t *hist = nullptr;
    uint32_t sort_blocks = 0;

    // host staging (host_buffers mode), grown on demand
    float *st_f = nullptr, *st_fhat = nullptr, *st_g = nullptr;
    uint64_t st_cap_v = 0;
    EditRec *st_edits = nullptr;
    uint64_t st_cap_edits = 0;
    // sequence staging (exactz_ws_correct_sequence): two slots of inputs and
    // outputs, a copy-in and a copy-out stream, grown on first use
    float *sq_f[2] = {}, *sq_fhat[2] = {}, *sq_g[2] = {};
    EditRec *sq_edits[2] = {};
    uint64_t sq_cap_v = 0, sq_cap_edits = 0;
    cudaStream_t sq_in = nullptr, sq_out = nullptr;
    cudaEvent_t sq_start = nullptr, sq_in_ev[2] = {}, sq_out_ev[2] = {};

    FieldState *h_fst = nullptr;  // pinned host copy
    LoopState *h_ls = nullptr;

    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;  // graph capture: the pass body forks in two
    cudaEvent_t cap_fork = nullptr, cap_join = nullptr;
    cudaStream_t aux = nullptr;  // the edit list, beside the residual check
    cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[6] = {0, 0, 0, 0, 0, 0};
    uint64_t layout_hash = 0;  // dims of the previous run (padding must hold k = 0, no CP bits)
    uint64_t tile_field_key = 0;  // layout the tile-field table was filled for
    exactz_stats stats{};
    cudaEvent_t ev[9] = {};
    cudaEvent_t kev[4] = {};  // around the loop kernels of one host-driven pass (profiling)
    Tuning tun;

    // extremum-graph lists of the original event constraints, grown on demand
    uint32_t *ev_E = nullptr;  // path ends (set-up scratch), one per arena vertex
    uint32_t *ev_start = nullptr;
    uint16_t *ev_cnt = nullptr;
    uint32_t *ev_list = nullptr;
    uint32_t *ev_radj = nullptr;
    uint32_t *ev_room = nullptr;                 // list room per 32 words of the listed-point bitmap
    unsigned long long *ev_room_off = nullptr;   // its exclusive prefix sums
    uint8_t *ev_tdone = nullptr;                 // per tile: every path end found
    float *refl = nullptr;                       // increasing edits: the reflected -f and -f_hat
    float *g_mirror = nullptr;                   // padded copies of g (fields whose rows are not 16-byte multiples)
    uint64_t cap_mirror = 0;
    uint64_t ev_cap[9] = {};  // E, start, cnt, list, radj, room, room_off, tdone, refl (elements)
    // set by the allocation-free entry point: every buffer is carved from its
    // fixed scratch, and a request to grow one fails with EXACTZ_ENOMEM
    // instead of allocating; alloc_refused counts such requests
    bool no_alloc = false;
    uint64_t alloc_refused = 0;

    std::mutex mu;
};

namespace {

template <class T>
int dalloc(exactz_workspace *ws, T *&p, uint64_t count)
{
    if (ws->no_alloc) {
        ws->alloc_refused++;
        return EXACTZ_ENOMEM;
    }
    if (count == 0) count = 1;
    void *q = nullptr;
    if (dev_malloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return EXACTZ_ENOMEM;
    }
    ws->allocs.push_back(q);
    ws->bytes += count * sizeof(T);
    p = static_cast<T *>(q);
    return EXACTZ_OK;
}

void free_ws(exactz_workspace *ws)
{
    if (ws->gexec) cudaGraphExecDestroy(ws->gexec);
    if (ws->graph) cudaGraphDestroy(ws->graph);
    if (ws->cap_stream) cudaStreamDestroy(ws->cap_stream);
    if (ws->cap_stream2) cudaStreamDestroy(ws->cap_stream2);
    if (ws->cap_fork) cudaEventDestroy(ws->cap_fork);
    if (ws->cap_join) cudaEventDestroy(ws->cap_join);
    if (ws->aux) cudaStreamDestroy(ws->aux);
    if (ws->aux_fork) cudaEventDestroy(ws->aux_fork);
    if (ws->aux_join) cudaEventDestroy(ws->aux_join);
    for (cudaEvent_t e : ws->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ws->kev)
        if (e) cudaEventDestroy(e);
    for (void *p : ws->allocs) cudaFree(p);
    void *ev[9] = {ws->ev_E,    ws->ev_start, ws->ev_cnt,      ws->ev_list, ws->ev_radj,
                   ws->ev_room, ws->ev_room_off, ws->ev_tdone, ws->refl};
    for (void *p : ev)
        if (p) cudaFree(p);
    if (ws->st_f) cudaFree(ws->st_f);
    if (ws->st_fhat) cudaFree(ws->st_fhat);
    if (ws->st_g) cudaFree(ws->st_g);
    if (ws->st_edits) cudaFree(ws->st_edits);
    if (ws->sq_in) cudaStreamSynchronize(ws->sq_in);
    if (ws->sq_out) cudaStreamSynchronize(ws->sq_out);
    for (int b = 0; b < 2; b++) {
        for (void *p : {(void *)ws->sq_f[b], (void *)ws->sq_fhat[b], (void *)ws->sq_g[b], (void *)ws->sq_edits[b]})
            if (p) cudaFree(p);
        if (ws->sq_in_ev[b]) cudaEventDestroy(ws->sq_in_ev[b]);
        if (ws->sq_out_ev[b]) cudaEventDestroy(ws->sq_out_ev[b]);
    }
    if (ws->sq_start) cudaEventDestroy(ws->sq_start);
    if (ws->sq_in) cudaStreamDestroy(ws->sq_in);
    if (ws->sq_out) cudaStreamDestroy(ws->sq_out);
    if (ws->h_fst) cudaFreeHost(ws->h_fst);
    if (ws->h_ls) cudaFreeHost(ws->h_ls);
    delete ws;
}

#define CK(x)                                                  \
    do {                                                       \
        cudaError_t e_ = (x);                                  \
        if (e_ != cudaSuccess) {                               \
            if (getenv("EXACTZ_DEBUG"))                        \
                fprintf(stderr, "exactz: %s at %s:%d\n",       \
                        cudaGetErrorString(e_), __FILE__, __LINE__); \
            cudaGetLastError();                                \
            return e_ == cudaErrorMemoryAllocation ? EXACTZ_ENOMEM : EXACTZ_ENODEV; \
        }                                                      \
    } while (0)

int ws_alloc(exactz_workspace *ws, const Layout &L)
{
    std::call_once(g_multi_once, build_multi_table);
    CK(cudaGetDevice(&ws->device));
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    ws->cap_nf = L.nfields;
    ws->cap_v = L.total_v;
    ws->cap_w = L.total_w;
    ws->cap_real = L.total_real;
    ws->cap_tiles = L.total_tiles;
    ws->sort_blocks = (uint32_t)nsm * 2;
    const uint64_t V = L.total_v, W = L.total_w, T = L.total_tiles, C = L.total_real;
    const uint64_t nblk = std::max(V / VBLOCK, W / WBLOCK) + 1;
    int rc = EXACTZ_OK;
#define AL(p, n) \
    if ((rc = dalloc(ws, p, n)) != EXACTZ_OK) return rc
    AL(ws->d_fields, L.nfields);
    AL(ws->d_fst, L.nfields);
    AL(ws->d_ls, 1);
    AL(ws->d_multi, 512);
    AL(ws->desc, V);
    AL(ws->cp_rank, V);
    AL(ws->cpwords, W);
    AL(ws->reqw, W);
    AL(ws->dirty, W);
    AL(ws->gs, C);
    AL(ws->pairbits, 3 * ((C + 31) / 32) + 1);  // pair bits, then the event and pinned event bits
    AL(ws->apply_flag, T);
    AL(ws->tile_flag, T);
    AL(ws->pin_tile_arena, T);
    AL(ws->pin_tile_bits, T / 32 + 1);
    AL(ws->pin_pair_arena, 2 * C);
    AL(ws->fids, L.nfields);
    if (L.nfields > 1) AL(ws->tile_field, L.total_tiles);
    if (L.total_mirror) {
        AL(ws->g_mirror, L.total_mirror);
        ws->cap_mirror = L.total_mirror;
    }
    AL(ws->d_tmaps, (uint64_t)TMAPS * L.nfields);
    AL(ws->cp_key[0], C);
    AL(ws->cp_key[1], C);
    AL(ws->cp_ent[0], C);
    AL(ws->cp_ent[1], C);
    AL(ws->blk, nblk);
    AL(ws->blk_off, nblk);
    AL(ws->hist, 256ull * ws->sort_blocks);
#undef AL
    CK(cudaMemcpy(ws->d_multi, g_multi_host, sizeof(g_multi_host), cudaMemcpyHostToDevice));
    CK(cudaMemset(ws->desc, 0, V * 4));
    {
        std::vector<uint32_t> ids(L.nfields);
        for (uint32_t i = 0; i < L.nfields; i++) ids[i] = i;
        CK(cudaMemcpy(ws->fids, ids.data(), 4ull * L.nfields, cudaMemcpyHostToDevice));
    }
    CK(cudaMemset(ws->cpwords, 0, W * 4));
    CK(cudaMemset(ws->reqw, 0, W * 4));
    CK(cudaMemset(ws->dirty, 0, W * 4));
    CK(cudaMallocHost(&ws->h_fst, sizeof(FieldState) * L.nfields));
    CK(cudaMallocHost(&ws->h_ls, sizeof(LoopState)));
    CK(cudaStreamCreateWithFlags(&ws->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ws->cap_stream2, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ws->cap_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ws->cap_join, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&ws->aux, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ws->aux_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ws->aux_join, cudaEventDisableTiming));
    for (cudaEvent_t &e : ws->ev) CK(cudaEventCreate(&e));
    for (cudaEvent_t &e : ws->kev) CK(cudaEventCreate(&e));
    return EXACTZ_OK;
}

Dev make_dev(exactz_workspace *ws, const Layout &L)
{
    Dev D{};
    D.fields = ws->d_fields;
    D.tmaps = ws->d_tmaps;
    D.fst = ws->d_fst;
    D.ls = ws->d_ls;
    D.nfields = L.nfields;
    D.total_tiles = L.total_tiles;
    D.total_v = L.total_v;
    D.total_w = L.total_w;
    D.desc = ws->desc;
    D.cp_rank = ws->cp_rank;
    D.cpwords = ws->cpwords;
    D.reqw = ws->reqw;
    D.dirty = ws->dirty;
    D.gs = ws->gs;
    D.pairbits = ws->pairbits;
    D.apply_flag = ws->apply_flag;
    D.tile_flag = ws->tile_flag;
    D.pin_tile_bits = ws->pin_tile_bits;
    D.cp_key[0] = ws->cp_key[0];
    D.cp_key[1] = ws->cp_key[1];
    D.cp_ent[0] = ws->cp_ent[0];
    D.cp_ent[1] = ws->cp_ent[1];
    D.o = ws->cp_ent[sort_passes(0, L.nfields) & 1];
    D.multi = ws->d_multi;
    D.cp_cap = ws->cap_real;
    D.blk = ws->blk;
    D.blk_off = ws->blk_off;
    D.hist = ws->hist;
    D.sort_blocks = ws->sort_blocks;
    D.tun = ws->tun;
    return D;
}

// Graph: [loop-flag kernel] -> while (flag) { check, pairs, apply, bookkeeping },
// the body as four kernels or (fused) as one cooperative kernel.
int ensure_graph(exactz_workspace *ws, const Dev &D, bool fused)
{
    uint64_t evk = D.events ^ (fused ? 0x8000000000000000ull : 0ull);
    for (const void *p : {(const void *)D.ev_start, (const void *)D.ev_cnt, (const void *)D.ev_list,
                          (const void *)D.ev_radj})
        evk = (evk ^ (uint64_t)(uintptr_t)p) * 1099511628211ull;
    const uint64_t key[6] = {D.nfields, D.total_tiles, D.total_v, D.total_w,
                             (uint64_t)(uintptr_t)D.o ^ ((uint64_t)D.tun.stencil_bps << 48) ^
                                 ((uint64_t)D.tun.apply_bps << 40) ^ ((uint64_t)D.tun.pairs_bps << 32) ^
                                 ((uint64_t)D.tun.chunked << 56),
                             evk};
    if (ws->gexec && std::memcmp(key, ws->gkey, sizeof(key)) == 0) return EXACTZ_OK;
    if (ws->gexec) {
        cudaGraphExecDestroy(ws->gexec);
        ws->gexec = nullptr;
    }
    if (ws->graph) {
        cudaGraphDestroy(ws->graph);
        ws->graph = nullptr;
    }
    cudaStream_t cs = ws->cap_stream;
    unsigned pgrid = 0;
    if (fused) CK(pass_grid(&pgrid));
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    ws->graph = g;
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_loop_flag(D, h, 1, cs);
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &nd));
    // the params union has no default constructor: zero raw storage instead
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    CK(cudaGraphAddNode(&cn, g, deps, nullptr, nd, &cp));
    CK(cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaStreamEndCapture(cs, &g));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (fused) {
        CK(launch_pass(D, h, pgrid, cs));
    } else {
        // the vertex check and the CP-pair check read nothing the other writes
        // (both only OR request bits and set apply flags): they run side by side
        CK(cudaEventRecord(ws->cap_fork, cs));
        CK(cudaStreamWaitEvent(ws->cap_stream2, ws->cap_fork, 0));
        launch_pairs_list(D, ws->cap_stream2);
        CK(cudaEventRecord(ws->cap_join, ws->cap_stream2));
        launch_check_list(D, cs);
        CK(cudaStreamWaitEvent(cs, ws->cap_join, 0));
        launch_apply(D, 1, cs);
        launch_book(D, h, 1, cs);
    }
    CK(cudaStreamEndCapture(cs, &body));
    CK(cudaGraphInstantiate(&ws->gexec, g, 0));
    std::memcpy(ws->gkey, key, sizeof(key));
    return EXACTZ_OK;
}

int grow_staging(exactz_workspace *ws, uint64_t V, uint64_t E)
{
    if (ws->no_alloc && (V > ws->st_cap_v || E > ws->st_cap_edits)) {
        ws->alloc_refused++;
        return EXACTZ_ENOMEM;
    }
    if (V > ws->st_cap_v) {
        if (ws->st_f) cudaFree(ws->st_f);
        if (ws->st_fhat) cudaFree(ws->st_fhat);
        if (ws->st_g) cudaFree(ws->st_g);
        ws->st_f = ws->st_fhat = ws->st_g = nullptr;
        ws->st_cap_v = 0;
        CK(dev_malloc(&ws->st_f, V * 4));
        CK(dev_malloc(&ws->st_fhat, V * 4));
        CK(dev_malloc(&ws->st_g, V * 4));
        ws->st_cap_v = V;
    }
    if (E > ws->st_cap_edits) {
        if (ws->st_edits) cudaFree(ws->st_edits);
        ws->st_edits = nullptr;
        ws->st_cap_edits = 0;
        CK(dev_malloc(&ws->st_edits, E * sizeof(EditRec)));
        ws->st_cap_edits = E;
    }
    return EXACTZ_OK;
}

// Two slots of sequence staging for fields of V vertices and E edit records,
// plus the copy streams and their events (created once).
int grow_sequence(exactz_workspace *ws, uint64_t V, uint64_t E)
{
    if (ws->no_alloc) {
        ws->alloc_refused++;
        return EXACTZ_ENOMEM;
    }
    if (!ws->sq_in) {
        CK(cudaStreamCreateWithFlags(&ws->sq_in, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&ws->sq_out, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ws->sq_start, cudaEventDisableTiming));
        for (int b = 0; b < 2; b++) {
            CK(cudaEventCreateWithFlags(&ws->sq_in_ev[b], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ws->sq_out_ev[b], cudaEventDisableTiming));
        }
    }
    if (V > ws->sq_cap_v) {
        for (int b = 0; b < 2; b++) {
            for (float **p : {&ws->sq_f[b], &ws->sq_fhat[b], &ws->sq_g[b]}) {
                if (*p) cudaFree(*p);
                *p = nullptr;
            }
        }
        ws->sq_cap_v = 0;
        for (int b = 0; b < 2; b++) {
            CK(dev_malloc(&ws->sq_f[b], V * 4));
            CK(dev_malloc(&ws->sq_fhat[b], V * 4));
            CK(dev_malloc(&ws->sq_g[b], V * 4));
        }
        ws->sq_cap_v = V;
    }
    if (E > ws->sq_cap_edits) {
        for (int b = 0; b < 2; b++) {
            if (ws->sq_edits[b]) cudaFree(ws->sq_edits[b]);
            ws->sq_edits[b] = nullptr;
        }
        ws->sq_cap_edits = 0;
        for (int b = 0; b < 2; b++) CK(dev_malloc(&ws->sq_edits[b], E * sizeof(EditRec)));
        ws->sq_cap_edits = E;
    }
    return EXACTZ_OK;
}

// Grow one event buffer (index i of ws->ev_cap) to `need` elements; contents are not kept.
template <class T>
int ev_grow(exactz_workspace *ws, T *&p, int i, uint64_t need)
{
    if (need == 0) need = 1;
    if (need <= ws->ev_cap[i]) return EXACTZ_OK;
    if (ws->no_alloc) {
        ws->alloc_refused++;
        return EXACTZ_ENOMEM;
    }
    if (p) cudaFree(p);
    p = nullptr;
    ws->bytes -= ws->ev_cap[i] * sizeof(T);
    ws->ev_cap[i] = 0;
    CK(dev_malloc(&p, need * sizeof(T)));
    ws->ev_cap[i] = need;
    ws->bytes += need * sizeof(T);
    return EXACTZ_OK;
}

// Extremum graph of f for the original event constraints (Sec. 4.2): per
// listed saddle the extrema its integral paths reach and their EGP selection,
// per linked extremum the saddles it is linked to.  Runs after the sort (the
// listed saddles and their positions are known); synchronises the stream to
// follow the pointer jumping and to size the lists.
int event_setup(exactz_workspace *ws, Dev &D, const Layout &L, cudaStream_t s, uint64_t &launches)
{
    int rc;
    LoopState *dls = ws->d_ls;
    LoopState *hls = ws->h_ls;
    CK(cudaMemcpyAsync(hls, dls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t nq = hls->total_cp;
    const uint64_t nchunks = (L.total_w + 31) / 32;
    if ((rc = ev_grow(ws, ws->ev_E, 0, 2 * L.total_v)) || (rc = ev_grow(ws, ws->ev_start, 1, nq)) ||
        (rc = ev_grow(ws, ws->ev_cnt, 2, nq)) || (rc = ev_grow(ws, ws->ev_room, 5, nchunks)) ||
        (rc = ev_grow(ws, ws->ev_room_off, 6, nchunks)) || (rc = ev_grow(ws, ws->ev_tdone, 7, L.total_tiles)))
        return rc;
    D.ev_start = ws->ev_start;
    D.ev_cnt = ws->ev_cnt;
    CK(cudaMemsetAsync(ws->ev_tdone, 0, L.total_tiles, s));
    // room for the lists (no path is followed yet), while the links are set up
    launch_ev_lists(D, nullptr, 0, ws->ev_room, nullptr, nullptr, nullptr, nullptr, s);
    launch_scan_u32(ws->ev_room, ws->ev_room_off, nchunks, &dls->ev_cursor[0], s);
    launch_ev_init(D, ws->ev_E, s);
    launches += 3;
    // pointer jumping: each round at least doubles the distance covered, so
    // every path within a field ends within 64 rounds
    for (int rounds = 0;; rounds++) {
        if (rounds == 64) return EXACTZ_ENODEV;
        CK(cudaMemsetAsync(&dls->ev_changed, 0, sizeof(uint32_t), s));
        launch_ev_jump(D, ws->ev_E, ws->ev_tdone, s);
        launches++;
        CK(cudaMemcpyAsync(hls, dls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!hls->ev_changed) break;
    }
    const uint64_t room = hls->ev_cursor[0];
    if (room >= (1ull << 32)) return EXACTZ_ESIZE;
    if ((rc = ev_grow(ws, ws->ev_list, 3, room))) return rc;
    D.ev_list = ws->ev_list;
    launch_ev_lists(D, ws->ev_E, 1, nullptr, ws->ev_room_off, ws->ev_list, ws->ev_start, ws->ev_cnt, s);
    CK(cudaMemcpyAsync(hls, dls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t entries = hls->ev_cursor[1];
    if (2 * entries + 1 >= (1ull << 32)) return EXACTZ_ESIZE;
    if ((rc = ev_grow(ws, ws->ev_radj, 4, 2 * entries + 1))) return rc;
    D.ev_radj = ws->ev_radj;
    launch_ev_reverse(D, ws->ev_radj, s);
    launches += 3;
    CK(cudaGetLastError());
    return EXACTZ_OK;
}

// after_launch, if set, is called once this call has queued its own uploads
// (graph loops, which read nothing back until they end) or once its
// host-driven loop is done: the batch sequence queues the next step's bulk
// copies there, so that they hold up none of this call's small copies.
int run(exactz_workspace *ws, uint32_t nf, const float *const *f, const float *const *fhat,
        const exactz_dims *d, const float *xi, const exactz_opts *o, float *const *g_out,
        exactz_edit *const *edits_out, const uint64_t *caps, exactz_result *res, cudaStream_t s,
        int host, const std::function<bool()> &after_launch = {})
{
    exactz_opts opt;
    exactz_default_opts(&opt);
    if (o) opt = *o;
    if (opt.N < 1 || opt.N > 254 || opt.mode > EXACTZ_MODE_FUSED || opt.events > EXACTZ_EVENTS_ORIGINAL ||
        opt.direction > EXACTZ_EDITS_INCREASING)
        return EXACTZ_EINVAL;
    const bool events = opt.events == EXACTZ_EVENTS_ORIGINAL;
    const bool inc = opt.direction == EXACTZ_EDITS_INCREASING;
    if (!f || !fhat || !d || !xi || !g_out || !res) return EXACTZ_EINVAL;
    Layout L;
    int rc = make_layout(nf, d, L);
    if (rc) return rc;
    for (uint32_t i = 0; i < nf; i++) {
        if (!f[i] || !fhat[i] || !g_out[i]) return EXACTZ_EINVAL;
        if (!(xi[i] > 0.0f) || !std::isfinite(xi[i])) return EXACTZ_EINVAL;
    }
    if (nf > ws->cap_nf || L.total_v > ws->cap_v || L.total_w > ws->cap_w || L.total_tiles > ws->cap_tiles ||
        L.total_real > ws->cap_real)
        return EXACTZ_ESIZE;
    if (events) {  // 31-bit arena indices in the path ends, 32-bit positions in the event lists
        if (L.total_v >= (1ull << 31)) return EXACTZ_ESIZE;
    }
    CK(cudaSetDevice(ws->device));

    uint64_t ecap_total = 0;
    std::vector<uint64_t> ebase(nf, 0);
    for (uint32_t i = 0; i < nf; i++) {
        ebase[i] = ecap_total;
        if (edits_out && edits_out[i] && caps) ecap_total += caps[i];
    }
    if (host) {
        if ((rc = grow_staging(ws, L.total_v, ecap_total)) != EXACTZ_OK) return rc;
    }
    if (inc && (rc = ev_grow(ws, ws->refl, 8, 2 * L.total_v)) != EXACTZ_OK) return rc;
    for (uint32_t i = 0; i < nf; i++) {
        FieldDesc &F = L.fd[i];
        F.N = opt.N;
        F.xi = xi[i];
        F.delta = xi[i] / (float)opt.N;  // binary32 division, Sec. 3.3
        F.max_iters = opt.max_iters;
        F.pin_tiles = ws->pin_tile_arena + F.tbase;
        F.pin_pairs = ws->pin_pair_arena + 2 * L.cpc[i];
        const bool has_edits = opt.want_edit_list && edits_out && edits_out[i] && caps && caps[i] > 0;
        F.edits_cap = has_edits ? caps[i] : 0;
        if (host) {
            float *sf = ws->st_f + F.vbase, *sh = ws->st_fhat + F.vbase;
            CK(cudaMemcpyAsync(sf, f[i], F.n * 4, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(sh, fhat[i], F.n * 4, cudaMemcpyHostToDevice, s));
            F.f = sf;
            F.fhat = sh;
            F.g = ws->st_g + F.vbase;
            F.edits = has_edits ? ws->st_edits + ebase[i] : nullptr;
        } else {
            F.f = f[i];
            F.fhat = fhat[i];
            F.g = g_out[i];
            F.edits = has_edits ? reinterpret_cast<EditRec *>(edits_out[i]) : nullptr;
        }
        if (inc) {  // correct the reflection of -f, -f_hat with decreasing edits
            float *rf = ws->refl + F.vbase, *rh = ws->refl + L.total_v + F.vbase;
            launch_reflect_in(F.f, rf, F.n, s);
            launch_reflect_in(F.fhat, rh, F.n, s);
            F.f = rf;
            F.fhat = rh;
            F.mirror = 1;
        }
    }
    if (ws->d_tmaps) {  // tile loads by TMA where the fields allow it
        std::vector<CUtensorMap> maps((uint64_t)TMAPS * nf);
        for (uint32_t i = 0; i < nf; i++) {
            FieldDesc &F = L.fd[i];
            CUtensorMap *m = &maps[(uint64_t)TMAPS * i];
            F.tma = (make_map(m, F.f, F, true) && make_map(m + 1, F.fhat, F, true) ? TMA_SETUP : 0u) |
                    (make_map(m + 3, ws->desc + F.vbase, F, false) ? TMA_DESC : 0u);
            if (make_map(m + 2, F.g, F, true)) {
                F.tma |= TMA_G;
            } else if (ws->g_mirror && L.mpitch[i] && L.total_mirror <= ws->cap_mirror) {  // the checks read a padded copy of g
                F.gm = ws->g_mirror + L.moff[i];
                F.pitch = L.mpitch[i];
                if (make_map(m + 2, F.gm, F, true, F.pitch)) F.tma |= TMA_G;
                else F.gm = nullptr;
            }
            if (getenv("EXACTZ_DEBUG")) fprintf(stderr, "exactz: field %u tile loads by TMA: %x\n", i, F.tma);
        }
        CK(cudaMemcpyAsync(ws->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice, s));
    }
    const uint64_t hsh = layout_key(nf, d);
    if (hsh != ws->layout_hash) {
        // a new layout: padding may hold another layout's vertices (edit counts, row bits)
        CK(cudaMemsetAsync(ws->desc, 0, L.total_v * 4, s));
        CK(cudaMemsetAsync(ws->cpwords, 0, L.total_w * 4, s));
        CK(cudaMemsetAsync(ws->reqw, 0, L.total_w * 4, s));
        CK(cudaMemsetAsync(ws->dirty, 0, L.total_w * 4, s));
        ws->layout_hash = hsh;
    }
    CK(cudaMemcpyAsync(ws->d_fields, L.fd.data(), sizeof(FieldDesc) * nf, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ws->d_fst, 0, sizeof(FieldState) * nf, s));
    CK(cudaMemsetAsync(ws->d_ls, 0, sizeof(LoopState), s));
    CK(cudaMemsetAsync(ws->tile_flag, 0, L.total_tiles, s));
    CK(cudaMemsetAsync(ws->pin_tile_bits, 0, (L.total_tiles / 32 + 1) * 4, s));
    CK(cudaMemsetAsync(ws->pairbits, 0, (events ? 3 * ((ws->cap_real + 31) / 32) + 1 : L.total_real / 32 + 1) * 4, s));
    CK(cudaMemsetAsync(ws->apply_flag, 0, L.total_tiles, s));
    // the graph loop reads nothing back before it ends (the event set-up does,
    // once per pointer-jumping round): the caller's bulk copies may start now,
    // behind this call's uploads
    const bool in_graph = opt.mode == EXACTZ_MODE_GRAPH || opt.mode == EXACTZ_MODE_FUSED;
    const bool early_hook = in_graph && !events;
    if (early_hook && after_launch && !after_launch()) return EXACTZ_ENODEV;
    Dev D = make_dev(ws, L);
    D.events = events ? 1u : 0u;
    if (nf > 1 && ws->tile_field) {  // the field of each tile: one load instead of a search over the fields
        if (ws->tile_field_key != hsh) {
            std::vector<uint32_t> tf(L.total_tiles);
            for (uint32_t i = 0; i < nf; i++) {
                const uint64_t t0 = L.fd[i].tbase, nt = (uint64_t)L.fd[i].tnx * L.fd[i].tny * L.fd[i].tnz;
                for (uint64_t t = 0; t < nt; t++) tf[t0 + t] = i;
            }
            CK(cudaMemcpy(ws->tile_field, tf.data(), 4ull * L.total_tiles, cudaMemcpyHostToDevice));
            ws->tile_field_key = hsh;
        }
        D.tile_field = ws->tile_field;
    }
    const int frontier = opt.mode != EXACTZ_MODE_PLAIN;
    const bool prof = opt.profile != 0;
    auto mark = [&](int i) {
        if (prof) cudaEventRecord(ws->ev[i], s);
    };
    const uint64_t P = (uint64_t)sort_passes(0, nf);
    const SetupRange R{0, L.total_tiles, 0, L.total_w / WBLOCK, 0, nf, 0, &ws->d_ls->total_cp};
    const FieldSet FS{ws->fids, nf, 0, L.total_v / VBLOCK, 0, nf};
    uint64_t launches = 0, loop_passes = 0;
    double loop_ms[3] = {0.0, 0.0, 0.0};

    // set-up and the first pass
    mark(0);
    launch_setup(D, R, s);
    mark(1);
    launch_cp_compact(D, R, s);
    mark(2);
    launch_cp_sort(D, R, s);
    if (events && (rc = event_setup(ws, D, L, s, launches)) != EXACTZ_OK) return rc;
    mark(3);
    launch_pairs_all(D, R, s);
    launch_apply(D, frontier, s);
    launch_book(D, 0, 0, s);
    mark(4);
    launches += 1 + 4 + 3 * P + 3;
    CK(cudaGetLastError());

    if (in_graph) {
        if ((rc = ensure_graph(ws, D, opt.mode == EXACTZ_MODE_FUSED)) != EXACTZ_OK) return rc;
        CK(cudaGraphLaunch(ws->gexec, s));
        launches += 1;  // loop-flag kernel; the body's kernels per pass are added below
        if (!early_hook && after_launch && !after_launch()) return EXACTZ_ENODEV;
    } else {
        for (;;) {
            CK(cudaMemcpyAsync(ws->h_ls, ws->d_ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (prof && loop_passes) {  // the previous pass's kernels have run
                for (int k = 0; k < 3; k++) {
                    float t = 0.0f;
                    cudaEventElapsedTime(&t, ws->kev[k], ws->kev[k + 1]);
                    loop_ms[k] += t;
                }
            }
            if (!ws->h_ls->any_active || ws->h_ls->fault) break;
            if (prof) cudaEventRecord(ws->kev[0], s);
            if (opt.mode == EXACTZ_MODE_PLAIN) launch_check_all(D, s);
            else launch_check_list(D, s);
            if (prof) cudaEventRecord(ws->kev[1], s);
            if (opt.mode == EXACTZ_MODE_PLAIN) launch_pairs_all(D, R, s);
            else launch_pairs_list(D, s);
            if (prof) cudaEventRecord(ws->kev[2], s);
            launch_apply(D, opt.mode == EXACTZ_MODE_PLAIN ? 0 : 1, s);
            if (prof) cudaEventRecord(ws->kev[3], s);
            launch_book(D, 0, 0, s);
            launches += 4;
            loop_passes++;
            CK(cudaGetLastError());
        }
        // (after the loop: its per-pass state reads never wait behind bulk copies)
        if (after_launch && !after_launch()) return EXACTZ_ENODEV;
    }
    mark(5);
    bool padded = false;
    for (uint32_t i = 0; i < nf; i++) padded = padded || L.fd[i].gm;
    // residual violations on pinned vertices and status; beside them g of the
    // fields kept in padded copies copied back (the residual check reads g from
    // those copies), then the edit list (the edit counts are final; the
    // residual check writes only request bits, flags and counters that neither
    // reads)
    cudaStream_t es = ws->aux ? ws->aux : s;
    if (es != s) {
        CK(cudaEventRecord(ws->aux_fork, s));
        CK(cudaStreamWaitEvent(es, ws->aux_fork, 0));
    }
    if (padded) launch_unmirror(D, es);
    launch_edit_list(D, FS, opt.want_edit_list ? 1 : 0, es);
    launch_check_pinned(D, FS, s);
    launch_pairs_pinned(D, FS, s);
    launch_finish(D, FS, s);
    mark(6);
    if (es != s) {
        CK(cudaEventRecord(ws->aux_join, es));
        CK(cudaStreamWaitEvent(s, ws->aux_join, 0));
    }
    if (inc)  // g back in the caller's coordinates and sign
        for (uint32_t i = 0; i < nf; i++) launch_reflect_out(L.fd[i].g, ws->desc + L.fd[i].vbase, L.fd[i].n, s);
    mark(7);
    launches += 4 + (padded ? 1 : 0) + (opt.want_edit_list ? 3 : 1) + (inc ? 3 * nf : 0);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ws->h_fst, ws->d_fst, sizeof(FieldState) * nf, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ws->h_ls, ws->d_ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ws->h_ls->fault) return EXACTZ_ENODEV;  // a halo load never completed
    std::memset(&ws->stats, 0, sizeof(ws->stats));
    ws->stats.passes = ws->h_ls->pass;
    ws->stats.total_critical = ws->h_ls->total_cp;
    ws->stats.sum_requests = ws->h_ls->sum_requests;
    ws->stats.sum_tiles = ws->h_ls->sum_tiles;
    ws->stats.sum_pairs = ws->h_ls->sum_pairs;
    ws->stats.sum_visits = ws->h_ls->sum_visits;
    if (in_graph)
        launches += (opt.mode == EXACTZ_MODE_FUSED ? 1 : 4) * (ws->h_ls->pass > 0 ? ws->h_ls->pass - 1 : 0);
    ws->stats.kernel_launches = launches;
    ws->stats.loop_passes = loop_passes;
    for (int k = 0; k < 3; k++) ws->stats.loop_kernel_ms[k] = (float)loop_ms[k];
    if (prof) {
        for (int i = 0; i < 7; i++) cudaEventElapsedTime(&ws->stats.stage_ms[i], ws->ev[i], ws->ev[i + 1]);
        cudaEventElapsedTime(&ws->stats.stage_ms[7], ws->ev[0], ws->ev[7]);
    }

    int ret = EXACTZ_OK;
    for (uint32_t i = 0; i < nf; i++) {
        const FieldState &S = ws->h_fst[i];
        exactz_result &R = res[i];
        std::memset(&R, 0, sizeof(R));
        R.iterations = S.iterations;
        R.n_edits = S.n_edits;
        R.n_lossless = S.n_lossless;
        R.residual_violations = S.capped + S.pinned_res;
        R.n_critical = events ? S.ncp_all : S.ncp;
        R.status = (int32_t)S.status;
        if (R.status < 0 && ret == EXACTZ_OK) ret = R.status;
        if (L.fd[i].edits && S.n_edits > L.fd[i].edits_cap && ret == EXACTZ_OK) ret = EXACTZ_ECAP;
    }
    if (host) {
        for (uint32_t i = 0; i < nf; i++) {
            const FieldDesc &F = L.fd[i];
            CK(cudaMemcpyAsync(g_out[i], F.g, F.n * 4, cudaMemcpyDeviceToHost, s));
            if (F.edits) {
                const uint64_t ne = std::min<uint64_t>(ws->h_fst[i].n_edits, F.edits_cap);
                if (ne)
                    CK(cudaMemcpyAsync(edits_out[i], F.edits, ne * sizeof(EditRec), cudaMemcpyDeviceToHost, s));
            }
        }
        CK(cudaStreamSynchronize(s));
    }
    return ret;
}

int check_device()
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return EXACTZ_ENODEV;
    }
    return EXACTZ_OK;
}

}  // namespace

// Allocation-failure injection (a testing aid): after `skip` more successful
// allocations, the next `count` fail as out of memory.
static std::mutex g_fail_mu;
static uint64_t g_fail_skip = 0, g_fail_left = 0;

cudaError_t exz::dev_malloc_bytes(void **p, size_t bytes)
{
    {
        std::lock_guard<std::mutex> lk(g_fail_mu);
        if (g_fail_left > 0) {
            if (g_fail_skip > 0) {
                g_fail_skip--;
            } else {
                g_fail_left--;
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
        }
    }
    return cudaMalloc(p, bytes);
}

extern "C" int exactz_debug_fail_allocations(uint64_t skip, uint64_t count)
{
    std::lock_guard<std::mutex> lk(g_fail_mu);
    g_fail_skip = skip;
    g_fail_left = count;
    return EXACTZ_OK;
}

const uint32_t *exz::host_multi_table()
{
    std::call_once(g_multi_once, build_multi_table);
    return g_multi_host;
}

// TMA tensor maps of the tile loads: a halo box of HXP x HY x HZ floats (NaN
// outside the field) of f, f_hat or g, or the tile's TX x TY x TZ descriptors.  The box's x coordinate is always 16-byte aligned
// (x0 - XOFF); the map needs rows of a multiple of 16 bytes (nx % 4 == 0) and a
// 16-byte aligned base.  Returns false (the field keeps the cp.async halo
// loads) where a map cannot be made.
bool exz::make_map(CUtensorMap *map, const void *base, const FieldDesc &F, bool halo, uint32_t pitch)
{
    if (!pitch) pitch = F.nx;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && fn)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else if (getenv("EXACTZ_DEBUG"))
            fprintf(stderr, "exactz: cuTensorMapEncodeTiled not found (%d, %d)\n", (int)e, (int)q);
        cudaGetLastError();
    });
    if (!encode || !base || (pitch % 4) != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) {
        if (getenv("EXACTZ_DEBUG"))
            fprintf(stderr, "exactz: no halo map (encoder %s, nx %u, base %p)\n", encode ? "found" : "missing", F.nx,
                    (const void *)base);
        return false;
    }
    const cuuint64_t dims[3] = {F.nx, F.ny, F.nz};
    const cuuint64_t strides[2] = {4ull * pitch, 4ull * pitch * F.ny};
    const cuuint32_t box[3] = {halo ? (cuuint32_t)HXP : (cuuint32_t)TX, halo ? (cuuint32_t)HY : (cuuint32_t)TY,
                               halo ? (cuuint32_t)HZ : (cuuint32_t)TZ};
    const cuuint32_t elem[3] = {1, 1, 1};
    const CUresult r = encode(map, halo ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
                              const_cast<void *>(base), dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              halo ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS && getenv("EXACTZ_DEBUG"))
        fprintf(stderr, "exactz: halo map encoding failed (%d) for %u x %u x %u\n", (int)r, F.nx, F.ny, F.nz);
    return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- C ABI
extern "C" {

void exactz_default_opts(exactz_opts *o)
{
    if (!o) return;
    o->N = 5;
    o->mode = EXACTZ_MODE_GRAPH;
    o->max_iters = 1000000;
    o->want_edit_list = 1;
    o->profile = 0;
    o->events = EXACTZ_EVENTS_REFORMULATED;
    o->direction = EXACTZ_EDITS_DECREASING;
}

exactz_workspace *exactz_workspace_create(uint32_t nfields, const exactz_dims *dims)
{
    if (check_device() != EXACTZ_OK) return nullptr;
    Layout L;
    if (make_layout(nfields, dims, L) != EXACTZ_OK) return nullptr;
    exactz_workspace *ws = new (std::nothrow) exactz_workspace();
    if (!ws) return nullptr;
    if (ws_alloc(ws, L) != EXACTZ_OK) {
        free_ws(ws);
        return nullptr;
    }
    return ws;
}

void exactz_workspace_destroy(exactz_workspace *ws)
{
    if (ws) free_ws(ws);
}

uint64_t exactz_workspace_bytes(const exactz_workspace *ws) { return ws ? ws->bytes : 0; }

int exactz_ws_stats(const exactz_workspace *ws, exactz_stats *out)
{
    if (!ws || !out) return EXACTZ_EINVAL;
    *out = ws->stats;
    return EXACTZ_OK;
}

int exactz_ws_correct(exactz_workspace *ws, uint32_t nfields, const float *const *f, const float *const *fhat,
                      const exactz_dims *d, const float *xi, const exactz_opts *opts, float *const *g_out,
                      exactz_edit *const *edits_out, const uint64_t *edits_cap, exactz_result *res,
                      void *cuda_stream, int host_buffers)
{
    if (!ws) return EXACTZ_EINVAL;
    std::lock_guard<std::mutex> lk(ws->mu);
    return run(ws, nfields, f, fhat, d, xi, opts, g_out, edits_out, edits_cap, res,
               static_cast<cudaStream_t>(cuda_stream), host_buffers);
}

int exactz_ws_correct_batch_sequence(exactz_workspace *ws, uint32_t nsteps, uint32_t nfields, const exactz_dims *dims,
                                     const float *const *f, const float *const *fhat, const float *xi,
                                     const exactz_opts *opts, float *const *g_out, exactz_edit *const *edits_out,
                                     const uint64_t *edits_cap, exactz_result *res, void *cuda_stream)
{
    if (!ws || !dims || !f || !fhat || !xi || !g_out || !res || nfields == 0) return EXACTZ_EINVAL;
    exactz_opts opt;
    exactz_default_opts(&opt);
    if (opts) opt = *opts;
    if (opt.N < 1 || opt.N > 254 || opt.mode > EXACTZ_MODE_FUSED || opt.events > EXACTZ_EVENTS_ORIGINAL ||
        opt.direction > EXACTZ_EDITS_INCREASING)
        return EXACTZ_EINVAL;
    Layout L;
    if (int rc = make_layout(nfields, dims, L)) return rc;
    const uint64_t items = (uint64_t)nsteps * nfields;
    // each field's edit records have one region in a slot, sized for its largest cap over the steps
    std::vector<uint64_t> eoff(nfields + 1, 0);
    for (uint64_t i = 0; i < items; i++) {
        if (!f[i] || !fhat[i] || !g_out[i]) return EXACTZ_EINVAL;
        if (!(xi[i] > 0.0f) || !std::isfinite(xi[i])) return EXACTZ_EINVAL;
    }
    for (uint32_t j = 0; j < nfields; j++) {
        uint64_t cap = 0;
        for (uint32_t st = 0; st < nsteps; st++) {
            const uint64_t i = (uint64_t)st * nfields + j;
            if (edits_out && edits_out[i] && edits_cap) cap = std::max<uint64_t>(cap, edits_cap[i]);
        }
        eoff[j + 1] = eoff[j] + cap;
    }
    std::memset(res, 0, sizeof(exactz_result) * items);
    if (nsteps == 0) return EXACTZ_OK;
    std::lock_guard<std::mutex> lk(ws->mu);
    CK(cudaSetDevice(ws->device));
    if (int rc = grow_sequence(ws, L.total_v, opt.want_edit_list ? eoff[nfields] : 0)) return rc;
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the copies in start after the caller's earlier work on its stream
    CK(cudaEventRecord(ws->sq_start, s));
    CK(cudaStreamWaitEvent(ws->sq_in, ws->sq_start, 0));
    auto copy_in = [&](uint32_t st) -> bool {
        const int b = (int)(st & 1u);
        for (uint32_t j = 0; j < nfields; j++) {
            const uint64_t i = (uint64_t)st * nfields + j, n = L.fd[j].n, v = L.fd[j].vbase;
            if (cudaMemcpyAsync(ws->sq_f[b] + v, f[i], n * 4, cudaMemcpyHostToDevice, ws->sq_in) != cudaSuccess ||
                cudaMemcpyAsync(ws->sq_fhat[b] + v, fhat[i], n * 4, cudaMemcpyHostToDevice, ws->sq_in) !=
                    cudaSuccess)
                return false;
        }
        return cudaEventRecord(ws->sq_in_ev[b], ws->sq_in) == cudaSuccess;
    };
    std::vector<const float *> fi(nfields), hi(nfields);
    std::vector<float *> gi(nfields);
    std::vector<exactz_edit *> ei(nfields);
    std::vector<uint64_t> ci(nfields);
    int ret = copy_in(0) ? EXACTZ_OK : EXACTZ_ENODEV;
    for (uint32_t st = 0; st < nsteps && (ret == EXACTZ_OK || ret == EXACTZ_ECAP); st++) {
        const int b = (int)(st & 1u);
        const uint64_t i0 = (uint64_t)st * nfields;
        // this slot's inputs have landed and its outputs (step st - 2) have left
        if (cudaStreamWaitEvent(s, ws->sq_in_ev[b], 0) != cudaSuccess ||
            cudaStreamWaitEvent(s, ws->sq_out_ev[b], 0) != cudaSuccess) {
            ret = EXACTZ_ENODEV;
            break;
        }
        for (uint32_t j = 0; j < nfields; j++) {
            const uint64_t i = i0 + j, v = L.fd[j].vbase;
            fi[j] = ws->sq_f[b] + v;
            hi[j] = ws->sq_fhat[b] + v;
            gi[j] = ws->sq_g[b] + v;
            const bool want = opt.want_edit_list && edits_out && edits_out[i] && edits_cap && edits_cap[i] > 0;
            ei[j] = want ? reinterpret_cast<exactz_edit *>(ws->sq_edits[b] + eoff[j]) : nullptr;
            ci[j] = want ? edits_cap[i] : 0;
        }
        // the next step's inputs go to the other slot, whose step (st - 1) is
        // finished, once this step's loop is queued: copies queued earlier
        // would hold up this step's own small uploads on the copy engine
        bool next_in = st + 1 >= nsteps;
        const auto queue_next = [&]() -> bool {
            next_in = true;
            return copy_in(st + 1);
        };
        const std::function<bool()> hook = st + 1 < nsteps ? std::function<bool()>(queue_next) : nullptr;
        int rc = run(ws, nfields, fi.data(), hi.data(), dims, &xi[i0], &opt, gi.data(), ei.data(), ci.data(),
                     &res[i0], s, 0, hook);
        if (rc == EXACTZ_OK || rc == EXACTZ_ECAP) {
            if (!next_in && !copy_in(st + 1)) rc = EXACTZ_ENODEV;  // run() ended before its loop
        }
        if (rc != EXACTZ_OK && rc != EXACTZ_ECAP) {
            ret = rc;
            break;
        }
        if (rc == EXACTZ_ECAP) ret = rc;
        // run() returned with the step finished: its results leave on the copy-out stream
        bool ok = true;
        for (uint32_t j = 0; j < nfields && ok; j++) {
            const uint64_t i = i0 + j;
            ok = cudaMemcpyAsync(g_out[i], gi[j], L.fd[j].n * 4, cudaMemcpyDeviceToHost, ws->sq_out) == cudaSuccess;
            const uint64_t ne = ei[j] ? std::min<uint64_t>(res[i].n_edits, ci[j]) : 0;
            if (ok && ne)
                ok = cudaMemcpyAsync(edits_out[i], ei[j], ne * sizeof(EditRec), cudaMemcpyDeviceToHost,
                                     ws->sq_out) == cudaSuccess;
        }
        if (!ok || cudaEventRecord(ws->sq_out_ev[b], ws->sq_out) != cudaSuccess) {
            ret = EXACTZ_ENODEV;
            break;
        }
    }
    const bool drained =
        cudaStreamSynchronize(ws->sq_in) == cudaSuccess && cudaStreamSynchronize(ws->sq_out) == cudaSuccess;
    if (!drained) {
        cudaGetLastError();
        if (ret == EXACTZ_OK || ret == EXACTZ_ECAP) ret = EXACTZ_ENODEV;
    }
    return ret;
}

int exactz_ws_correct_sequence(exactz_workspace *ws, uint32_t nitems, const float *const *f,
                               const float *const *fhat, exactz_dims d, const float *xi,
                               const exactz_opts *opts, float *const *g_out, exactz_edit *const *edits_out,
                               const uint64_t *edits_cap, exactz_result *res, void *cuda_stream)
{
    // a sequence of one-field batches
    return exactz_ws_correct_batch_sequence(ws, nitems, 1, &d, f, fhat, xi, opts, g_out, edits_out, edits_cap, res,
                                            cuda_stream);
}

int exactz_ws_get_tuning(const exactz_workspace *ws, exactz_tuning *out)
{
    if (!ws || !out) return EXACTZ_EINVAL;
    out->stencil_blocks_per_sm = ws->tun.stencil_bps;
    out->apply_blocks_per_sm = ws->tun.apply_bps;
    out->pairs_blocks_per_sm = ws->tun.pairs_bps;
    out->chunked_schedule = ws->tun.chunked;
    out->best_ms = 0.f;
    return EXACTZ_OK;
}

int exactz_ws_set_tuning(exactz_workspace *ws, const exactz_tuning *t)
{
    if (!ws || !t) return EXACTZ_EINVAL;
    if (t->stencil_blocks_per_sm < 1 || t->stencil_blocks_per_sm > 64 || t->apply_blocks_per_sm < 1 ||
        t->apply_blocks_per_sm > 64 || t->pairs_blocks_per_sm < 1 || t->pairs_blocks_per_sm > 64 ||
        t->chunked_schedule > 1)
        return EXACTZ_EINVAL;
    std::lock_guard<std::mutex> lk(ws->mu);
    ws->tun.stencil_bps = t->stencil_blocks_per_sm;
    ws->tun.apply_bps = t->apply_blocks_per_sm;
    ws->tun.pairs_bps = t->pairs_blocks_per_sm;
    ws->tun.chunked = t->chunked_schedule;
    return EXACTZ_OK;
}

// Coordinate descent over the launch schedule: each knob in turn takes every
// candidate value with the others fixed, and keeps the one whose whole
// correction of these fields ran fastest (CUDA events on the caller's stream,
// best of `repeats`).  The result never depends on the schedule.
int exactz_ws_autotune(exactz_workspace *ws, uint32_t nfields, const float *const *f, const float *const *fhat,
                       const exactz_dims *d, const float *xi, const exactz_opts *opts, void *cuda_stream,
                       uint32_t repeats, exactz_tuning *out)
{
    if (!ws || !out) return EXACTZ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<float *> gtmp(nfields, nullptr);
    std::vector<exactz_result> res(nfields);
    int rc = EXACTZ_OK;
    for (uint32_t i = 0; i < nfields && !rc; i++) {
        if (!d) { rc = EXACTZ_EINVAL; break; }
        const uint64_t n = (uint64_t)d[i].nx * d[i].ny * d[i].nz;
        if (dev_malloc(&gtmp[i], n * 4) != cudaSuccess) rc = EXACTZ_ENOMEM;
    }
    exactz_opts o;
    exactz_default_opts(&o);
    if (opts) o = *opts;
    o.want_edit_list = 0;
    o.profile = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = EXACTZ_ENODEV;
    auto time_one = [&](float &ms) -> int {
        ms = 1e30f;
        for (uint32_t r = 0; r < (repeats ? repeats : 2); r++) {
            cudaEventRecord(e0, s);
            int c = exactz_ws_correct(ws, nfields, f, fhat, d, xi, &o, gtmp.data(), nullptr, nullptr, res.data(),
                                      cuda_stream, 0);
            cudaEventRecord(e1, s);
            if (c != EXACTZ_OK && c != EXACTZ_ECAP) return c;
            if (cudaEventSynchronize(e1) != cudaSuccess) return EXACTZ_ENODEV;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        return EXACTZ_OK;
    };
    float best = 0.f;
    if (!rc) rc = time_one(best);  // also warms the graph and caches
    if (!rc) rc = time_one(best);
    // candidates per knob: blocks per SM of the check (10 resident), apply (4
    // resident) and pair kernels, and the schedule
    static const uint32_t cands[4][5] = {{6, 12, 24, 36, 48}, {4, 8, 16, 32, 0}, {2, 4, 8, 16, 0}, {0, 1, 0, 0, 0}};
    static const int ncand[4] = {5, 4, 4, 2};
    for (int knob = 0; knob < 4 && !rc; knob++) {
        const int nc = ncand[knob];
        Tuning keep = ws->tun;
        for (int c = 0; c < nc && !rc; c++) {
            Tuning cand = keep;
            if (knob == 0) cand.stencil_bps = cands[0][c];
            else if (knob == 1) cand.apply_bps = cands[1][c];
            else if (knob == 2) cand.pairs_bps = cands[2][c];
            else cand.chunked = cands[3][c];
            if (std::memcmp(&cand, &keep, sizeof(Tuning)) == 0) continue;
            {
                std::lock_guard<std::mutex> lk(ws->mu);
                ws->tun = cand;
            }
            float t = 0.f;
            rc = time_one(t);
            if (!rc && t < best) {
                best = t;
                keep = cand;
            }
        }
        std::lock_guard<std::mutex> lk(ws->mu);
        ws->tun = keep;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (float *p : gtmp)
        if (p) cudaFree(p);
    if (rc) return rc;
    exactz_ws_get_tuning(ws, out);
    out->best_ms = best;
    return EXACTZ_OK;
}

int exactz_correct_batch(uint32_t nfields, const float *const *f, const float *const *fhat, const exactz_dims *d,
                         const float *xi, const exactz_opts *opts, float *const *g_out,
                         exactz_edit *const *edits_out, const uint64_t *edits_cap, exactz_result *res,
                         void *cuda_stream)
{
    int rc = check_device();
    if (rc) return rc;
    Layout L;
    if ((rc = make_layout(nfields, d, L)) != EXACTZ_OK) return rc;
    exactz_workspace *ws = exactz_workspace_create(nfields, d);
    if (!ws) return EXACTZ_ENOMEM;
    rc = exactz_ws_correct(ws, nfields, f, fhat, d, xi, opts, g_out, edits_out, edits_cap, res, cuda_stream, 0);
    exactz_workspace_destroy(ws);
    return rc;
}

int exactz_correct(const float *f, const float *fhat, exactz_dims d, float xi, const exactz_opts *opts,
                   float *g_out, exactz_edit *edits_out, uint64_t edits_cap, exactz_result *res,
                   void *cuda_stream)
{
    const float *fp[1] = {f};
    const float *hp[1] = {fhat};
    float *gp[1] = {g_out};
    exactz_edit *ep[1] = {edits_out};
    uint64_t cp[1] = {edits_cap};
    return exactz_correct_batch(1, fp, hp, &d, &xi, opts, gp, ep, cp, res, cuda_stream);
}

int exactz_classify(const float *h, exactz_dims d, uint32_t *desc_out, uint8_t *type_out, void *cuda_stream)
{
    int rc = check_device();
    if (rc) return rc;
    if (!h || !desc_out) return EXACTZ_EINVAL;
    Layout L;
    if ((rc = make_layout(1, &d, L)) != EXACTZ_OK) return rc;
    exactz_workspace *ws = exactz_workspace_create(1, &d);
    if (!ws) return EXACTZ_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    L.fd[0].f = h;
    L.fd[0].fhat = h;
    L.fd[0].N = 5;
    rc = EXACTZ_OK;
    if (cudaMemcpyAsync(ws->d_fields, L.fd.data(), sizeof(FieldDesc), cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = EXACTZ_ENODEV;
    if (!rc) {
        launch_classify(make_dev(ws, L), desc_out, type_out, s);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = EXACTZ_ENODEV;
    }
    exactz_workspace_destroy(ws);
    return rc;
}

int exactz_cp_order(const float *f, exactz_dims d, uint64_t *order_out, uint64_t *count_out, void *cuda_stream)
{
    int rc = check_device();
    if (rc) return rc;
    if (!f || !order_out || !count_out) return EXACTZ_EINVAL;
    Layout L;
    if ((rc = make_layout(1, &d, L)) != EXACTZ_OK) return rc;
    exactz_workspace *ws = exactz_workspace_create(1, &d);
    if (!ws) return EXACTZ_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    float *scratch = nullptr;
    rc = EXACTZ_OK;
    if (dev_malloc(&scratch, L.fd[0].n * 4) != cudaSuccess) rc = EXACTZ_ENOMEM;
    if (!rc) {
        FieldDesc &F = L.fd[0];
        F.f = f;
        F.fhat = f;
        F.g = scratch;
        F.N = 5;
        F.xi = 1.0f;
        F.delta = 0.2f;
        F.pin_tiles = ws->pin_tile_arena;
        F.pin_pairs = ws->pin_pair_arena;
        const Dev D = make_dev(ws, L);
        const SetupRange R{0, L.total_tiles, 0, L.total_w / WBLOCK, 0, 1, 0, &ws->d_ls->total_cp};
        cudaMemcpyAsync(ws->d_fields, L.fd.data(), sizeof(FieldDesc), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(ws->d_fst, 0, sizeof(FieldState), s);
        cudaMemsetAsync(ws->d_ls, 0, sizeof(LoopState), s);
        launch_setup(D, R, s);
        launch_cp_compact(D, R, s);
        launch_cp_sort(D, R, s);
        cudaMemcpyAsync(ws->h_ls, ws->d_ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(ws->h_fst, ws->d_fst, sizeof(FieldState), cudaMemcpyDeviceToHost, s);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = EXACTZ_ENODEV;
        if (!rc && ws->h_fst[0].err) rc = (ws->h_fst[0].err & ERR_NONFINITE) ? EXACTZ_ENONFINITE : EXACTZ_EBOUND;
        if (!rc) {
            const uint64_t c = ws->h_ls->total_cp;
            *count_out = c;
            if (c && (cudaMemcpyAsync(order_out, D.o, c * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                      cudaStreamSynchronize(s) != cudaSuccess))
                rc = EXACTZ_ENODEV;
        }
    }
    if (scratch) cudaFree(scratch);
    exactz_workspace_destroy(ws);
    return rc;
}

const char *exactz_version(void)
{
    return "exactz-b300 0.2 (sm_103a; tile 32x8x4; stencil/sort/apply kernels; graph while-loop)";
}

// Scratch of the edit-stream calls: block counts, their offsets, the total
// and a "malformed" flag; freed on every return.
struct StreamScratch {
    uint32_t *blk = nullptr;
    unsigned long long *off = nullptr, *total = nullptr;
    int *bad = nullptr;
    ~StreamScratch()
    {
        if (blk) cudaFree(blk);
        if (off) cudaFree(off);
        if (total) cudaFree(total);
        if (bad) cudaFree(bad);
    }
    int alloc(uint64_t nb, cudaStream_t s)
    {
        CK(dev_malloc(&blk, 4 * (nb ? nb : 1)));
        CK(dev_malloc(&off, 8 * (nb ? nb : 1)));
        CK(dev_malloc(&total, 8));
        CK(dev_malloc(&bad, sizeof(int)));
        CK(cudaMemsetAsync(total, 0, 8, s));
        CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
        return EXACTZ_OK;
    }
    // the total and the flag, after the stream's work so far
    int read(cudaStream_t s, unsigned long long &t, int &b)
    {
        CK(cudaMemcpyAsync(&t, total, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&b, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return EXACTZ_OK;
    }
};

int exactz_encode_edits(const exactz_edit *edits, uint64_t n_edits, uint64_t n, uint32_t N, uint8_t *kcodes_out,
                        float *lossless_out, uint64_t lossless_cap, uint64_t *n_lossless_out, void *cuda_stream)
{
    int rc = check_device();
    if (rc) return rc;
    if (!kcodes_out || !n_lossless_out || (n_edits && !edits) || (lossless_cap && !lossless_out) || n == 0 ||
        N < 1 || N > 254)
        return EXACTZ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const EditRec *e = reinterpret_cast<const EditRec *>(edits);
    const uint64_t nb = stream_blocks(n_edits);
    StreamScratch S;
    if ((rc = S.alloc(nb, s))) return rc;
    CK(cudaMemsetAsync(kcodes_out, 0, n, s));
    launch_stream_kcodes(e, n_edits, n, N, kcodes_out, S.bad, s);
    launch_stream_count(e, nullptr, n_edits, N, 0, S.blk, S.bad, s);
    if (nb) launch_scan_u32(S.blk, S.off, nb, S.total, s);
    CK(cudaGetLastError());
    unsigned long long total = 0;
    int bad = 0;
    if ((rc = S.read(s, total, bad))) return rc;
    if (bad) return EXACTZ_EINVAL;
    *n_lossless_out = total;
    if (total > lossless_cap) return EXACTZ_ECAP;
    launch_stream_lossless(e, n_edits, S.off, lossless_out, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return EXACTZ_OK;
}

int exactz_decode_edits(const float *fhat, uint64_t n, float xi, uint32_t N, uint32_t direction,
                        const uint8_t *kcodes, const float *lossless, float *g_out, void *cuda_stream)
{
    int rc = check_device();
    if (rc) return rc;
    if (!fhat || !kcodes || !g_out || n == 0 || N < 1 || N > 254 || !(xi > 0.0f) || !std::isfinite(xi) ||
        direction > EXACTZ_EDITS_INCREASING)
        return EXACTZ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const uint64_t nb = stream_blocks(n);
    StreamScratch S;
    if ((rc = S.alloc(nb, s))) return rc;
    launch_stream_count(nullptr, kcodes, n, N, 1, S.blk, S.bad, s);
    launch_scan_u32(S.blk, S.off, nb, S.total, s);
    CK(cudaGetLastError());
    unsigned long long total = 0;
    int bad = 0;
    if ((rc = S.read(s, total, bad))) return rc;
    if (bad || (total && !lossless)) return EXACTZ_EINVAL;
    const float delta = xi / (float)N;  // binary32 division, Sec. 3.3
    launch_stream_decode(fhat, kcodes, lossless, n, N, delta, direction == EXACTZ_EDITS_INCREASING, S.off, g_out,
                         s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return EXACTZ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free entry point
// exactz_correct_noalloc: the same correction for small fields, with every
// device buffer carved out of one fixed array that lives in this library's
// device image.  It is for callers that cannot allocate device memory in the
// middle of their work: simulations and in-situ pipelines that reserve the
// whole device memory up front for their own pool (a cudaMalloc would fail or
// take memory they have promised elsewhere), and loops that cannot take the
// implicit device synchronisation of cudaMalloc / cudaFree.  The loop is
// driven from the host: every pass reads a few bytes of loop state back and
// synchronises the caller's stream, and the call returns only after its work
// on the stream has finished.
//
// The array is file-scope static device storage: every GPU that loads this
// library holds EXACTZ_NOALLOC_SCRATCH_BYTES of it until the process exits.
// In host code the symbol is only a host-side stand-in, so its device address
// is obtained once per device with cudaGetSymbolAddress (with that device
// current) on the first call there.  All calls share the array and it keeps
// the last call's contents, so each call clears what must start at zero.  Two
// calls whose GPU work overlapped would race on the shared array: calls from
// one process are serialised by a lock, and the lock is released only after
// the call's stream has drained, on error paths too.
namespace {

constexpr uint64_t kNoallocBytes = EXACTZ_NOALLOC_SCRATCH_BYTES;
constexpr uint64_t kNoallocMaxV = EXACTZ_NOALLOC_MAX_VERTICES;
constexpr uint32_t kNoallocSortBlocks = 512;  // at most 2 radix-sort blocks per SM for up to 256 SMs
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The pieces carved from the scratch array, in order, and their byte offsets
// (each piece starts on 256 bytes) for a layout of V arena vertices, W row
// words, T tiles, C critical-point slots, nf fields, nblk scan blocks and sb
// radix-sort blocks.  The roles are the ones ws_alloc gives the same buffers.
enum NoallocPiece {
    P_MULTI, P_FIELDS, P_FST, P_LS, P_DESC, P_CPRANK, P_CPWORDS, P_REQW, P_DIRTY, P_GS, P_PAIRBITS,
    P_APPLY, P_TILEFLAG, P_PINTILE, P_PINBITS, P_PINPAIR, P_FIDS, P_KEY0, P_KEY1, P_ENT0, P_ENT1,
    P_BLK, P_BLKOFF, P_HIST, P_REFL, P_COUNT
};
struct CarvePlan {
    uint64_t off[P_COUNT];
    uint64_t used;
};

constexpr CarvePlan carve_plan(uint64_t V, uint64_t W, uint64_t T, uint64_t C, uint64_t nf, uint64_t nblk,
                               uint64_t sb)
{
    const uint64_t bytes[P_COUNT] = {
        512 * 4,                       // link-component table
        nf * sizeof(FieldDesc), nf * sizeof(FieldState), sizeof(LoopState),
        4 * V, 4 * V,                  // descriptors, CP ranks
        4 * W, 4 * W, 4 * W,           // CP, request and dirty row words
        4 * C, 4 * (C / 32 + 1),       // sorted CP values, pair bits
        T, T, 4 * T, 4 * (T / 32 + 1), // apply / check flags, pinned tiles and their bits
        8 * C, 4 * nf,                 // pinned pairs, field ids
        4 * C, 4 * C, 8 * C, 8 * C,    // radix-sort keys and entries (ping-pong)
        4 * nblk, 8 * nblk, 4 * 256 * sb,  // block counts, offsets, digit histograms
        8 * V};                        // increasing edits: the reflected -f and -f_hat
    CarvePlan p{};
    uint64_t used = 0;
    for (int i = 0; i < P_COUNT; i++) {
        const uint64_t off = (used + 255) / 256 * 256;
        p.off[i] = off;
        used = off + (bytes[i] ? bytes[i] : 1);
    }
    p.used = used;
    return p;
}

// The largest field the call accepts fits: a field of n <= kNoallocMaxV
// vertices has V = round_up(n, VBLOCK) <= kNoallocMaxV arena vertices, at most
// n row words (a row of nx vertices has ceil(nx / 32) <= nx words), at most n
// tiles and n critical-point slots (about 72 bytes per vertex in all).
static_assert(kNoallocMaxV % VBLOCK == 0 && kNoallocMaxV % WBLOCK == 0, "padding of the largest field");
static_assert(carve_plan(kNoallocMaxV, kNoallocMaxV, kNoallocMaxV, kNoallocMaxV, 1,
                         kNoallocMaxV / WBLOCK + 1, kNoallocSortBlocks)
                      .used <= kNoallocBytes,
              "the largest accepted field must fit the fixed scratch");

struct NoallocDevice {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch on this device
};

NoallocDevice g_noalloc_dev[kNoallocMaxDevices];
exactz_workspace g_noalloc_ws[kNoallocMaxDevices];  // static host objects, no device allocation
FieldState g_noalloc_hfst[kNoallocMaxDevices];      // pageable host read-back buffers
LoopState g_noalloc_hls[kNoallocMaxDevices];
std::mutex g_noalloc_mu;

// Point every workspace buffer for layout L into the scratch array.
bool noalloc_carve(exactz_workspace *ws, unsigned char *base, const Layout &L, int nsm)
{
    const uint64_t V = L.total_v, W = L.total_w, T = L.total_tiles, C = L.total_real;
    const uint64_t nblk = std::max(V / VBLOCK, W / WBLOCK) + 1;
    ws->sort_blocks = std::min<uint32_t>((uint32_t)nsm * 2, kNoallocSortBlocks);
    const CarvePlan p = carve_plan(V, W, T, C, L.nfields, nblk, ws->sort_blocks);
    if (p.used > kNoallocBytes) return false;
    auto at = [&](auto *&ptr, int piece) {
        ptr = reinterpret_cast<std::remove_reference_t<decltype(ptr)>>(base + p.off[piece]);
    };
    at(ws->d_multi, P_MULTI);
    at(ws->d_fields, P_FIELDS);
    at(ws->d_fst, P_FST);
    at(ws->d_ls, P_LS);
    at(ws->desc, P_DESC);
    at(ws->cp_rank, P_CPRANK);
    at(ws->cpwords, P_CPWORDS);
    at(ws->reqw, P_REQW);
    at(ws->dirty, P_DIRTY);
    at(ws->gs, P_GS);
    at(ws->pairbits, P_PAIRBITS);
    at(ws->apply_flag, P_APPLY);
    at(ws->tile_flag, P_TILEFLAG);
    at(ws->pin_tile_arena, P_PINTILE);
    at(ws->pin_tile_bits, P_PINBITS);
    at(ws->pin_pair_arena, P_PINPAIR);
    at(ws->fids, P_FIDS);
    at(ws->cp_key[0], P_KEY0);
    at(ws->cp_key[1], P_KEY1);
    at(ws->cp_ent[0], P_ENT0);
    at(ws->cp_ent[1], P_ENT1);
    at(ws->blk, P_BLK);
    at(ws->blk_off, P_BLKOFF);
    at(ws->hist, P_HIST);
    at(ws->refl, P_REFL);
    ws->ev_cap[8] = 2 * V;  // run() finds the reflection storage in place
    ws->cap_nf = L.nfields;
    ws->cap_v = V;
    ws->cap_w = W;
    ws->cap_real = C;
    ws->cap_tiles = L.total_tiles;
    ws->bytes = p.used;
    ws->no_alloc = true;  // any request to grow a buffer fails instead of allocating
    return true;
}

// Drains the call's stream when the call returns (on every path), before the
// lock on the shared scratch is released.
struct StreamDrain {
    cudaStream_t s;
    ~StreamDrain()
    {
        if (cudaStreamSynchronize(s) != cudaSuccess) cudaGetLastError();
    }
};

}  // namespace

extern "C" int exactz_correct_noalloc(const float *f, const float *fhat, exactz_dims d, float xi,
                                      const exactz_opts *opts, float *g_out, exactz_edit *edits_out,
                                      uint64_t edits_cap, exactz_result *res, void *cuda_stream)
{
    int rc = check_device();
    if (rc) return rc;
    if (!f || !fhat || !g_out || !res) return EXACTZ_EINVAL;
    // the event lists need storage sized after the sort (the reflected fields
    // of increasing edits fit in the fixed scratch)
    if (opts && (opts->events != EXACTZ_EVENTS_REFORMULATED || opts->direction > EXACTZ_EDITS_INCREASING))
        return EXACTZ_EINVAL;
    Layout L;
    if ((rc = make_layout(1, &d, L)) != EXACTZ_OK) return rc;
    if (L.total_real > EXACTZ_NOALLOC_MAX_VERTICES) return EXACTZ_ESIZE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return EXACTZ_ENODEV;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    const StreamDrain drain{s};  // destroyed first: the stream drains before the lock is released
    NoallocDevice &D = g_noalloc_dev[dev];
    exactz_workspace *ws = &g_noalloc_ws[dev];
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (!D.ready) {
        // set-up, once per device: the device address of the static array
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return EXACTZ_ENODEV;
        }
        D.base = static_cast<unsigned char *>(p);
        std::call_once(g_multi_once, build_multi_table);
        D.ready = true;
    }
    if (!noalloc_carve(ws, D.base, L, nsm)) return EXACTZ_ESIZE;
    ws->device = dev;
    ws->h_fst = &g_noalloc_hfst[dev];
    ws->h_ls = &g_noalloc_hls[dev];
    // the array keeps the previous call's contents: reset what must start at zero
    static const uint32_t zero_fid = 0;
    if (cudaMemcpyAsync(ws->d_multi, g_multi_host, sizeof(g_multi_host), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ws->fids, &zero_fid, sizeof(zero_fid), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(ws->desc, 0, L.total_v * 4, s) != cudaSuccess ||
        cudaMemsetAsync(ws->reqw, 0, L.total_w * 4, s) != cudaSuccess ||
        cudaMemsetAsync(ws->cpwords, 0, L.total_w * 4, s) != cudaSuccess ||
        cudaMemsetAsync(ws->dirty, 0, L.total_w * 4, s) != cudaSuccess) {
        cudaGetLastError();
        return EXACTZ_ENODEV;
    }
    ws->layout_hash = layout_key(1, &d);  // cleared above: run() need not clear them again
    // no graph objects or events here: the loop is driven from the host
    exactz_opts opt;
    exactz_default_opts(&opt);
    if (opts) opt = *opts;
    if (opt.mode == EXACTZ_MODE_GRAPH || opt.mode == EXACTZ_MODE_FUSED) opt.mode = EXACTZ_MODE_FRONTIER;
    opt.profile = 0;
    const float *fp[1] = {f};
    const float *hp[1] = {fhat};
    float *gp[1] = {g_out};
    exactz_edit *ep[1] = {edits_out};
    uint64_t cp[1] = {edits_cap};
    return run(ws, 1, fp, hp, &d, &xi, &opt, gp, ep, cp, res, s, 0);
}
