// exz_common.cuh -- shared device-side definitions of the B300 correction.
//
// Grid and order (EXaCTz Sec. 3, Sec. 3.3 footnote): vertices of an
// nx*ny*nz grid, index x + nx*(y + ny*z); neighbours are the 14 offsets of the
// Freudenthal triangulation (every component in {0,1}, or every component in
// {0,-1}); ties in value are broken by vertex index.  The closed
// neighbourhood of a vertex is listed by "rank" 0..14 in increasing vertex
// index (rank 7 is the vertex itself), which is the lexicographic order of
// the offsets by (dz, dy, dx).  A running arg-max with ">=" (arg-min with "<")
// over ranks in that order therefore implements the index tie-break.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace exz {

// ---------------------------------------------------------------- geometry
constexpr int TX = 32;   // tile width: one warp per tile row, one cp-bitmap word
constexpr int TY = 8;
constexpr int TZ = 4;
constexpr int TILE_V = TX * TY * TZ;
// Halo tile in shared memory: HY x HZ rows of HXP floats.  Slot j of a row
// holds x = x0 - XOFF + j, so x0 - 1 .. x0 + TX sit at slots XOFF - 1 .. XOFF + TX
// and the TX tile values start on a 16-byte boundary.  The whole halo is the
// box of one TMA tile load (cp.async.bulk.tensor) whose x coordinate, x0 - XOFF,
// is 16-byte aligned; cells outside the field read as NaN.
constexpr int XOFF = 4;
constexpr int HXP = TX + 2 * XOFF;
constexpr int HY = TY + 2;
constexpr int HZ = TZ + 2;
constexpr int HALO_N = HXP * HY * HZ;
static_assert(HXP % 4 == 0 && XOFF >= 1 && XOFF % 4 == 0, "halo rows, tile values and the TMA x coordinate on 16 bytes");
static_assert((HALO_N * 4) % 128 == 0, "consecutive halo buffers keep the 128-byte alignment of TMA destinations");
constexpr int TMAPS = 4;  // tensor maps per field: f, f_hat, g, descriptors
constexpr int CTA = 256;
constexpr int WARPS = CTA / 32;
constexpr int ROWS = TY * TZ;
constexpr int VBLOCK = 4096;  // arena alignment of a field (vertices) = edit-list block
constexpr int WBLOCK = 2048;  // cp-bitmap alignment of a field (words) = compaction block
constexpr uint64_t LOCAL_BITS = 40;
constexpr uint64_t LOCAL_MASK = (1ull << LOCAL_BITS) - 1;

// offset (dx, dy, dz) of rank r; rank 14 - r is the opposite offset
__host__ __device__ constexpr int rdx(int r)
{
    return r == 7 ? 0 : (r < 7 ? ((r & 1) ? 0 : -1) : (((14 - r) & 1) ? 0 : 1));
}
__host__ __device__ constexpr int rdy(int r)
{
    return r == 7 ? 0 : (r < 7 ? (((r >> 1) & 1) ? 0 : -1) : ((((14 - r) >> 1) & 1) ? 0 : 1));
}
__host__ __device__ constexpr int rdz(int r)
{
    return r == 7 ? 0 : (r < 7 ? (r < 4 ? -1 : 0) : ((14 - r) < 4 ? 1 : 0));
}
// mask bit of rank r (r != 7) and the inverse
__host__ __device__ constexpr int slot_of(int r) { return r < 7 ? r : r - 1; }
__host__ __device__ constexpr int rank_of(int s) { return s < 7 ? s : s + 1; }
// smem offset of rank r inside a halo tile
__host__ __device__ constexpr int soff(int r) { return rdx(r) + HXP * rdy(r) + HXP * HY * rdz(r); }

// Descriptor bits (per vertex): steepest up / down rank and lower-link mask of
// f, the saddle flag of f, the "listed" flag (the vertex is in the sorted list
// of critical points whose order is kept: every critical point of f, or only
// its saddles under the original event constraints), and in the top byte the
// vertex's edit count k (0..N, N+1 = pinned at the lossless bound).  A vertex
// is a maximum (minimum) of f iff its steepest up (down) rank is 7, itself.
constexpr uint32_t D_UP_SHIFT = 0, D_DN_SHIFT = 4, D_MASK_SHIFT = 8;
constexpr uint32_t D_SADDLE = 1u << 22;
constexpr uint32_t D_CP = 1u << 23;
constexpr uint32_t D_K_SHIFT = 24;
constexpr uint32_t D_F_MASK = 0x00FFFFFFu;

// Tile loads by TMA (FieldDesc::tma bits): the halos of f and f_hat (set-up),
// the halo of g (checks; from gm where the field has one) and the tile's
// descriptors (checks); the others are staged with cp.async.
constexpr uint32_t TMA_SETUP = 1, TMA_G = 2, TMA_DESC = 4;

// Field errors (FieldState::err bits)
constexpr uint32_t ERR_NONFINITE = 1, ERR_BOUND = 2;
// Status codes (match the C ABI)
constexpr int32_t ST_CONVERGED = 1, ST_STUCK = 2, ST_ITER_LIMIT = 3;

// Division of 32-bit values by a run-time invariant divisor d with one
// high multiply (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// t = hi32(n m), n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
    uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while ((1ull << l) < d) l++;
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f)
{
    const uint32_t t = __umulhi(n, f.m);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// ------------------------------------------------------------ field table
struct FieldDesc {
    uint32_t nx, ny, nz, N;
    uint64_t n;
    uint32_t tnx, tny, tnz;        // tiles per axis (tnx = cp-bitmap words per row)
    uint32_t mirror;               // 1: the field is the point reflection of -f (increasing edits)
    uint32_t tma;                  // TMA_* bits: which tile loads use the tensor maps Dev::tmaps[TMAPS * field slot ..]
    uint32_t pitch;                // row pitch (vertices) of gm
    uint64_t tbase;                // first global tile id
    uint64_t vbase;                // arena offset (vertices): k, desc, cp_rank, request bits
    uint64_t wbase;                // cp-bitmap offset (words)
    const float *f;
    const float *fhat;
    float *g;
    float *gm;                     // g with rows padded to 16 bytes (fields whose g has no tensor map), or null:
                                   // while it is set, g lives there until k_unmirror copies it into g
    float xi, delta;
    uint64_t max_iters;
    struct EditRec *edits;  // output edit list (device), may be null
    uint64_t edits_cap;
    uint32_t *pin_tiles;    // tiles around this field's pinned vertices (capacity: its tile count)
    uint32_t *pin_pairs;    // CP pairs next to its pinned critical points (capacity: 2 n)
    FastDiv div_nx, div_ny;    // x = t mod nx, row = t / nx, z = row / ny (fields below 2^32 vertices)
    FastDiv div_tnx, div_tny;  // the same for tile coordinates
};

// One applied edit; same layout as exactz_edit (16 bytes).
struct EditRec {
    uint64_t idx;
    float value;
    uint8_t k;
    uint8_t lossless;
    uint16_t reserved;
};

struct FieldState {
    unsigned long long iterations;
    unsigned long long cp_base;
    unsigned long long ncp;
    unsigned long long capped;      // unpinned requests left unapplied at the cap
    unsigned long long pinned_res;  // pinned vertices still requested at exit
    unsigned long long n_edits;
    unsigned long long n_lossless;
    unsigned long long pin_tile_count;
    unsigned long long pin_pair_count;
    unsigned long long ncp_all;     // critical points of f when only the saddles are listed
    uint32_t had_req, done, err, status;
};

struct LoopState {
    unsigned long long total_cp;
    unsigned long long sum_requests;  // requests applied or skipped, over all passes
    unsigned long long sum_tiles;     // tiles checked by frontier passes
    unsigned long long sum_pairs;     // CP pairs checked by frontier passes
    unsigned long long sum_visits;    // vertices checked by frontier passes
    unsigned long long ev_cursor[3];  // event-list set-up: minima and maxima list ends, saddle-list end
    uint32_t any_active;
    uint32_t pass;
    uint32_t fault;  // a bounded wait ran out (the call reports EXACTZ_ENODEV)
    uint32_t ev_changed;  // event-list set-up: a path end moved in the last jump round
    uint32_t bar_count, bar_gen;  // fused pass kernel: blocks arrived at the grid barrier; its generation
    uint32_t pass_done, pad0;     // fused pass kernel: blocks done with the apply this pass
};

// Launch schedule of the per-pass kernels (chosen by the autotuner): blocks per
// SM of the tile-check, tile-apply and CP-pair kernels, and whether a block (or
// warp) takes a contiguous chunk of the tile bitmap's words (1) or every
// grid-th word (0).
struct Tuning {
    uint32_t stencil_bps = 48, apply_bps = 32, pairs_bps = 8, chunked = 0;
};

// All device pointers of one workspace, passed to kernels by value.
struct Dev {
    const FieldDesc *fields;
    FieldState *fst;
    LoopState *ls;
    uint32_t nfields;
    uint32_t total_tiles;
    uint64_t total_v;   // arena vertices (padded)
    uint64_t total_w;   // row words (padded): one bit per vertex, one word per tile row
    uint32_t *desc;
    uint32_t *cp_rank;
    uint32_t *cpwords;   // critical points of f (row words)
    uint32_t *reqw;      // vertices requested this pass (row words)
    uint32_t *dirty;     // vertices whose closed star changed last pass (row words)
    float *gs;           // g of the critical points, in f's sorted order
    uint32_t *pairbits;  // CP pairs (q, q+1) to check next pass, bit q
    uint8_t *apply_flag;  // per tile: holds requested vertices (taken and cleared by the apply kernel)
    uint8_t *tile_flag;   // per tile: to check next pass (taken and cleared by the check kernel)
    uint32_t *pin_tile_bits;
    uint32_t *cp_key[2];
    unsigned long long *cp_ent[2];
    unsigned long long *o;  // sorted critical points (aliases one of cp_ent)
    const uint32_t *multi;  // 2^14-bit table: link subset has >= 2 components
    uint64_t cp_cap;
    // scratch for scans, histograms and block counts
    uint32_t *blk;
    unsigned long long *blk_off;
    uint32_t *hist;
    uint32_t sort_blocks;
    Tuning tun;
    const uint32_t *tile_field;  // field slot of each tile when fields are placed freely (else null)
    // Original event constraints (Sec. 4.2), events != 0: the sorted list holds
    // the saddles of f only (C2 on its adjacent pairs), and per listed saddle q
    // the extrema its integral paths reach in f (C3): ev_cnt[q] = number of
    // linked minima | maxima << 8 (a side with fewer than two counts 0);
    // ev_list[ev_start[q] ...] holds the minima, then the maxima (field-local
    // vertex indices, each side's f-selection of Extremum Graph Pairing first).
    // For a linked extremum e, cp_rank[e] = h > 0 points into ev_radj:
    // ev_radj[h] = its number of linked saddles, followed by their positions q.
    // In pairbits, the pair bits are followed by the event bits of the next
    // pass and the event bits of the residual check, one word range each.
    // TMA tensor maps of each field's f, f_hat, g (halo boxes) and descriptors
    // (tile boxes), TMAPS per field slot; used where FieldDesc::tma is set
    const CUtensorMap *tmaps;
    uint32_t events;
    const uint32_t *ev_start;
    const uint16_t *ev_cnt;
    const uint32_t *ev_list;
    const uint32_t *ev_radj;
};

// Fields set up together: tiles [tile0, tile1), compaction blocks
// [wblk0, wblk0 + nwblk) of the row-word bitmap, fields [fid0, fid1), and the
// critical points placed from position cp0 on, their number in *cp_count.
struct SetupRange {
    uint32_t tile0, tile1;
    uint64_t wblk0, nwblk;
    uint32_t fid0, fid1;
    uint64_t cp0;
    unsigned long long *cp_count;
};

// Fields finished together: ids fids[0..n), arena blocks [vblk0, vblk0 + nvblk).
struct FieldSet {
    const uint32_t *fids;
    uint32_t n;
    uint64_t vblk0, nvblk;
    uint32_t fid0, fid1;  // the arena blocks belong to fields [fid0, fid1), placed in order
};

// Tiles [beg, end) with stride `step` of a list of `count` tiles handled by this block.
__device__ __forceinline__ void tile_range(const Dev &D, unsigned long long count, unsigned long long &beg,
                                           unsigned long long &end, unsigned long long &step)
{
    if (D.tun.chunked) {
        const unsigned long long c = (count + gridDim.x - 1) / gridDim.x;
        beg = blockIdx.x * c;
        end = min(count, beg + c);
        step = 1;
    } else {
        beg = blockIdx.x;
        end = count;
        step = gridDim.x;
    }
}

// Positions beg, beg + step, ... (< end) of the n tiles handled by worker `w`
// of `nworkers` (a block or a warp): every nworkers-th tile, or a contiguous
// chunk with the chunked schedule.
__device__ __forceinline__ void work_range(const Dev &D, uint32_t n, uint32_t w, uint32_t nworkers, uint32_t &beg,
                                           uint32_t &end, uint32_t &step)
{
    if (D.tun.chunked) {
        const uint32_t c = (n + nworkers - 1) / nworkers;
        beg = (uint32_t)min((uint64_t)n, (uint64_t)w * c);
        end = (uint32_t)min((uint64_t)n, (uint64_t)beg + c);
        step = 1;
    } else {
        beg = w;
        end = n;
        step = nworkers;
    }
}

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint32_t field_of_tile(const Dev &D, uint32_t tile)
{
    if (D.tile_field) return D.tile_field[tile];
    uint32_t lo = 0, hi = D.nfields - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (D.fields[mid].tbase <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Order-preserving 32-bit key of a finite float; -0 and +0 get the same key.
__device__ __forceinline__ uint32_t fkey(float v)
{
    uint32_t u = __float_as_uint(v);
    if (u == 0x80000000u) u = 0;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ bool multi_bit(const uint32_t *tab, uint32_t s)
{
    return (tab[s >> 5] >> (s & 31)) & 1u;
}

// Saddle test from a lower-link mask and the valid-neighbour mask.
__device__ __forceinline__ bool is_saddle(const uint32_t *tab, uint32_t L, uint32_t valid)
{
    uint32_t U = valid & ~L;
    return L != 0 && U != 0 && (multi_bit(tab, L) || multi_bit(tab, U));
}

// Warp-wide tile marking: each lane with `want` marks `tile` in the bitmap, and
// the lanes that set a bit first append their tiles to the list with a single
// counter update for the whole warp.  All 32 lanes must call it.
__device__ __forceinline__ void warp_mark_tiles(bool want, uint32_t tile, uint32_t *bits, uint32_t *list,
                                                unsigned long long *count)
{
    bool fresh = false;
    if (want) {
        const uint32_t bit = 1u << (tile & 31);
        if (!(__ldcg(&bits[tile >> 5]) & bit)) fresh = !(atomicOr(&bits[tile >> 5], bit) & bit);
    }
    const uint32_t b = __ballot_sync(0xffffffffu, fresh);
    if (!b) return;
    const int lane = threadIdx.x & 31, leader = __ffs(b) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (fresh) list[base + __popc(b & ((1u << lane) - 1u))] = tile;
}

}  // namespace exz
