// exz_kernels.cu -- sm_103a kernels of the EXaCTz correction (Algorithm 1).
//
//   k_stencil<SETUP>      per-vertex descriptor of f (steepest up/down rank,
//                         lower link mask, saddle / critical flags; Sec. 3.2,
//                         Sec. 4.2), input validation, g := f_hat, k := 0, the
//                         critical-point bitmap and the first pass's checks.
//   k_stencil<CHECK_*>    EG constraints and saddle-link rule on the edited
//                         field g (Sec. 4.2) for every tile, the flagged tiles'
//                         dirty vertices (frontier) or the pinned tiles
//                         (residual); emits decrease requests.
//   k_cp_*, k_sort_*      ordered compaction of critical points; stable LSD
//                         radix sort by (field, value key) -> f's global CP
//                         order (Sec. 4.3).
//   k_pairs               reformulated event constraint: adjacent CP pairs
//                         whose g-order is reversed (Sec. 4.3).
//   k_apply_tiles         bounded monotone edit (Sec. 3.3) of each requested
//                         vertex once; dirty bits and tile flags of the next pass.
//   k_book, k_loop_flag   per-field convergence bookkeeping, device loop flag.
//   k_status              residual violations and final status.
//   k_edit_*              ordered compaction of the edit list.
//
// Requests are deduplicated by a bitmap of row words over the arena; a vertex
// is edited at most once per pass (synchronous semantics, Sec. 4.4 proof).
// Requests to pinned vertices (already at the lossless bound) may be set; the
// apply kernel leaves them unchanged and they do not keep the loop running.
// Tiles to check or to apply are flagged with plain byte stores (one byte per
// tile); the consuming kernel takes and clears the flags.
#include <cmath>
#include <cstdio>

#include "exz_common.cuh"
#include "exz_launch.h"

namespace exz {

enum { SM_SETUP = 0, SM_CHECK_ALL = 1, SM_CHECK_LIST = 2, SM_PINNED = 3, SM_CLASSIFY = 4 };

// Block-size assumptions of the kernels below.
static_assert(TX == 32, "one row word (and one warp) per tile row");
static_assert(CTA % 32 == 0 && ROWS <= 32, "tile-row prefix sums run in one warp");
// The tile-stencil kernel runs smaller blocks than the others, so that more
// tiles are in flight per SM (its time goes mostly to memory latency per tile).
constexpr int SCTA = 128, STWARPS = SCTA / 32;  // 12 blocks per SM: 40 registers, no spills
static_assert(SCTA % 32 == 0 && SCTA >= 32 && SCTA >= ROWS, "stencil blocks: whole warps, one thread per tile row");
static_assert(STWARPS == TZ && TY <= 32, "frontier check: warp w visits the dirty vertices of z-slab w");
static_assert(WBLOCK % CTA == 0 && VBLOCK % (4 * CTA) == 0, "compaction and edit-list blocks");
// Block sizes of the one-block scans and of the small grid-stride kernels.
// Every launch below passes the named block size of its kernel's
// __launch_bounds__ (a CPU test parses this file and checks each launch).
constexpr int SCAN_NT = 1024;
constexpr int SMALL_NT = 256;

__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// A value of the reflected field back in the caller's sign.  The increasing
// edit computes fl(g + Delta) or fl(f + xi), which are never -0 for positive
// Delta and xi, while the negated reflection of an exact zero is -0: edited
// values (k > 0) are given as +0 then.
__device__ __forceinline__ float unreflect(float v, uint32_t k)
{
    const float w = -v;
    return (k != 0 && w == 0.0f) ? 0.0f : w;
}

// ------------------------------------------------------------ requests
// A request is a bit in the row-word bitmap reqw (one 32-bit word per tile row,
// bit = x mod 32); setting it twice is harmless, which deduplicates requests.
// Every tile holding a requested vertex is queued once in the apply list.
//
// The check kernel requests each target where it finds it: one atomic OR into
// the target's row word and a byte store of its tile's apply flag (both
// idempotent), with no per-tile collection and so no block barrier.

__device__ __forceinline__ int nb_index(int ox, int oy, int oz) { return (ox + 1) + 3 * ((oy + 1) + 3 * (oz + 1)); }

// Flag the tiles of a 27-bit neighbourhood mask around `tile`; lane j of the
// calling warp handles neighbour j.  Flags are plain byte stores: setting one
// twice, or from several threads, leaves the same result.
__device__ __forceinline__ void warp_mark_nb_tiles(uint32_t nb, uint32_t tile, uint32_t tnx, uint32_t tny,
                                                   uint8_t *flags)
{
    const int j = threadIdx.x & 31;
    if (j < 27 && ((nb >> j) & 1u)) {
        const int ox = j % 3 - 1, oy = (j / 3) % 3 - 1, oz = j / 9 - 1;
        flags[(int64_t)tile + ox + (int64_t)tnx * (oy + (int64_t)tny * oz)] = 1;
    }
}

// The field constants a tile's request emission needs, held in registers (the
// FieldDesc lives in global memory, which the emission's atomics and stores
// might alias, so reading it inside the loop would reload it every time).
struct EmitGeo {
    uint32_t nx, ny, tnx, tny, N;
    uint64_t vbase, wbase, tbase;
};

// Offset + 1 (0, 1 or 2) along one axis of every rank, two bits per rank.
__host__ __device__ constexpr uint32_t rank_axis_bits(int axis)
{
    uint32_t m = 0;
    for (int r = 0; r < 15; r++) m |= (uint32_t)((axis == 0 ? rdx(r) : (axis == 1 ? rdy(r) : rdz(r))) + 1) << (2 * r);
    return m;
}

// Request the closed-star ranks in m of vertex (x, y, z) of field G (every
// rank in m names a vertex of the field).  PINNED keeps only targets already
// at the lossless bound (the residual count).
template <bool PINNED>
__device__ __forceinline__ void emit_targets(const Dev &D, const EmitGeo &G, uint32_t x, uint32_t y, uint32_t z,
                                             uint32_t m)
{
    constexpr uint32_t BX = rank_axis_bits(0), BY = rank_axis_bits(1), BZ = rank_axis_bits(2);
    while (m) {
        const int r = __ffs(m) - 1;
        m &= m - 1;
        const uint32_t X = x + ((BX >> (2 * r)) & 3u) - 1u, Y = y + ((BY >> (2 * r)) & 3u) - 1u,
                       Z = z + ((BZ >> (2 * r)) & 3u) - 1u;
        const uint64_t row = (uint64_t)Z * G.ny + Y;
        if (PINNED && (D.desc[G.vbase + row * G.nx + X] >> D_K_SHIFT) <= G.N) continue;
        atomicOr(&D.reqw[G.wbase + row * G.tnx + (X >> 5)], 1u << (X & 31));
        const uint32_t tile = (uint32_t)(G.tbase + (X >> 5) + (uint64_t)G.tnx * (Y / TY + (uint64_t)G.tny * (Z / TZ)));
        if (!D.apply_flag[tile]) D.apply_flag[tile] = 1;
    }
}

// Request vertex t of field F from outside a tile (the CP-pair check): set its
// request bit and return its tile, which the caller queues (warp_mark_tiles).
__device__ __forceinline__ uint32_t request_vertex(const Dev &D, const FieldDesc &F, uint64_t t)
{
    uint32_t x, row;
    if (F.n < (1ull << 32)) {
        row = fdiv((uint32_t)t, F.div_nx);
        x = (uint32_t)t - row * F.nx;
    } else {
        row = (uint32_t)(t / F.nx);
        x = (uint32_t)(t - (uint64_t)row * F.nx);
    }
    const uint32_t z = fdiv(row, F.div_ny), y = row - z * F.ny;
    atomicOr(&D.reqw[F.wbase + (uint64_t)row * F.tnx + (x >> 5)], 1u << (x & 31));
    return (uint32_t)(F.tbase + (x >> 5) + (uint64_t)F.tnx * (y / TY + (uint64_t)F.tny * (z / TZ)));
}

// ------------------------------------------------------------ stencil core
// Steepest-ascent / -descent rank and lower-link mask of the vertex at smem
// index c.  Out-of-domain cells hold NaN: never selected, never "lower".
struct Stn {
    uint32_t up, dn, mask, valid;
};

__device__ __forceinline__ Stn stencil15(const float *s, int c)
{
    float v[15];
#pragma unroll
    for (int r = 0; r < 15; r++) v[r] = s[c + soff(r)];
    float mx = -INFINITY, mn = INFINITY;
    uint32_t up = 7, dn = 7;
#pragma unroll
    for (int r = 0; r < 15; r++) {
        if (v[r] >= mx) { mx = v[r]; up = r; }
        if (v[r] < mn) { mn = v[r]; dn = r; }
    }
    const float cv = v[7];
    uint32_t mask = 0;
#pragma unroll
    for (int r = 0; r < 7; r++) mask |= (v[r] <= cv) ? (1u << r) : 0u;
#pragma unroll
    for (int r = 8; r < 15; r++) mask |= (v[r] < cv) ? (1u << (r - 1)) : 0u;
    return Stn{up, dn, mask, 0x3FFFu};
}

// Mask bits (slots) of the neighbours whose offset along `axis` (0 = x,
// 1 = y, 2 = z) is `sign`.
__host__ __device__ constexpr uint32_t slots_along(int axis, int sign)
{
    uint32_t m = 0;
    for (int r = 0; r < 15; r++) {
        if (r == 7) continue;
        const int o = axis == 0 ? rdx(r) : (axis == 1 ? rdy(r) : rdz(r));
        if (o == sign) m |= 1u << slot_of(r);
    }
    return m;
}

// Neighbours of vertex (x, y, z) that lie in an nx x ny x nz field, as mask
// slots.  (Out-of-field halo cells also hold NaN, which no compare selects,
// so the stencil needs no other change at the boundary.)
__device__ __forceinline__ uint32_t valid_slots(uint32_t x, uint32_t y, uint32_t z, uint32_t nx, uint32_t ny,
                                                uint32_t nz)
{
    uint32_t out = 0;
    if (x == 0) out |= slots_along(0, -1);
    if (x + 1 >= nx) out |= slots_along(0, 1);
    if (y == 0) out |= slots_along(1, -1);
    if (y + 1 >= ny) out |= slots_along(1, 1);
    if (z == 0) out |= slots_along(2, -1);
    if (z + 1 >= nz) out |= slots_along(2, 1);
    return 0x3FFFu & ~out;
}

// Rules R1 (steepest neighbours) and R2 (saddle links) at one vertex, as the
// set of closed-star ranks whose vertices must be decreased:
//   R1: up_g != up_f -> up_g;  down_g != down_f -> down_f;
//   R2 (saddle in f or g): for each neighbour whose order against the vertex
//       differs between f and g, whichever of the two is lower in f.
__device__ __forceinline__ uint32_t request_mask(const uint32_t *smulti, uint32_t d, const Stn &g)
{
    const uint32_t upf = d & 15u, dnf = (d >> 4) & 15u, mf = (d >> 8) & 0x3FFFu;
    uint32_t m = 0;
    if (g.up != upf) m |= 1u << g.up;
    if (g.dn != dnf) m |= 1u << dnf;
    const uint32_t diff = g.mask ^ mf;
    if (diff && ((d & D_SADDLE) || is_saddle(smulti, g.mask, g.valid))) {
        const uint32_t nb = diff & mf;  // the neighbour is the lower one in f
        m |= (nb & 0x7Fu) | ((nb & 0x3F80u) << 1);  // slot -> rank
        if (diff & ~mf) m |= 1u << 7;   // the vertex itself is the lower one
    }
    return m;
}

// Position of the n-th (0-based) set bit of m (m has more than n set bits).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n)
{
    int pos = 0, c = __popc(m & 0xFFFFu);
    if (n >= c) { n -= c; pos += 16; m >>= 16; }
    c = __popc(m & 0xFFu);
    if (n >= c) { n -= c; pos += 8; m >>= 8; }
    c = __popc(m & 0xFu);
    if (n >= c) { n -= c; pos += 4; m >>= 4; }
    c = __popc(m & 0x3u);
    if (n >= c) { n -= c; pos += 2; m >>= 2; }
    if (n >= (int)(m & 1u)) pos += 1;
    return pos;
}

// cp.async of one 4-byte word into shared memory (completes at the next wait).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// cp.async of 16 bytes (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// TMA tile loads completing on an mbarrier (transaction count in bytes).
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Wait for the completion of phase `parity`, a bounded number of tries;
// false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 22); i++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
// Order this thread's earlier shared-memory accesses before later TMA writes.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// The box of tensor map `map` at (x, y, z) into shared memory at dst (128-byte aligned).
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

constexpr uint32_t NO_TILE = 0xFFFFFFFFu;

// Position of a tile in its field.
struct TileGeo {
    uint32_t fid, tx;
    int x0, y0, z0;
};

__device__ __forceinline__ TileGeo tile_geo_of(const Dev &D, uint32_t tile, uint32_t fid)
{
    TileGeo G;
    G.fid = fid;
    const FieldDesc &F = D.fields[G.fid];
    const uint32_t lt = (uint32_t)(tile - F.tbase);
    const uint32_t rest = fdiv(lt, F.div_tnx);
    G.tx = lt - rest * F.tnx;
    const uint32_t tz = fdiv(rest, F.div_tny), ty = rest - tz * F.tny;
    G.x0 = (int)(G.tx * TX);
    G.y0 = (int)(ty * TY);
    G.z0 = (int)(tz * TZ);
    return G;
}

__device__ __forceinline__ TileGeo tile_geo(const Dev &D, uint32_t tile)
{
    return tile_geo_of(D, tile, field_of_tile(D, tile));
}

// A staged tile's position and the constants of its field, published in
// shared memory by the warp that stages it, so that the checking threads read
// them there instead of each loading the field table from global memory.
struct TileInfo {
    TileGeo G;
    uint32_t nx, ny, nz, tnx, tny, N;
    uint64_t vbase, wbase, tbase;
    float xi;
    float *g;
    float *gm;  // the padded copy of g, or null
    uint32_t pitch;
};

__device__ __forceinline__ TileInfo tile_info(const TileGeo &G, const FieldDesc &F)
{
    return TileInfo{G, F.nx, F.ny, F.nz, F.tnx, F.tny, F.N, F.vbase, F.wbase, F.tbase, F.xi, F.g, F.gm, F.pitch};
}

// One tile per block iteration: the tile's values plus a one-vertex halo are
// staged in shared memory (NaN outside the domain), then every vertex (SETUP,
// CHECK_ALL, PINNED, CLASSIFY) or every dirty vertex (CHECK_LIST) is checked.
// Tiles come from [t0, t1) (SETUP, CHECK_ALL, CLASSIFY), the set bits of
// tile_flag (CHECK_LIST, taken and cleared 32 candidates at a time), or the
// pinned-tile lists of fields fids[0..nf) (PINNED).
// The next tile is staged with cp.async into a second buffer while the
// current one is checked.
// (The body of k_stencil and of the fused pass kernel's check phase; blocks of
// SCTA threads.)
template <int MODE>
__device__ __forceinline__ void stencil_tiles(const Dev &D, uint32_t *desc_out, uint8_t *type_out, uint32_t t0,
                                              uint32_t t1, const uint32_t *fids, uint32_t nf)
{
    constexpr int NB = 2;
    __shared__ __align__(128) float sa[NB][HALO_N];
    __shared__ __align__(128) float sb[MODE == SM_SETUP ? NB : 1][MODE == SM_SETUP ? HALO_N : 32];
    __shared__ __align__(8) uint64_t s_mbar[NB];  // completion of each buffer's TMA loads
    constexpr bool CHECK = MODE == SM_CHECK_ALL || MODE == SM_CHECK_LIST || MODE == SM_PINNED;
    __shared__ __align__(128) uint32_t s_desc[NB][CHECK ? TILE_V : 32];  // the tile's descriptors (TMA fields)
    __shared__ uint32_t smulti[512];
    __shared__ uint32_t s_err, s_ncp;
    __shared__ uint32_t s_rw[NB][ROWS];   // dirty row words of the tile (CHECK_LIST)
    __shared__ uint16_t s_vis[MODE == SM_CHECK_LIST ? TILE_V : 1];  // the tile's dirty vertices (row << 5 | lx)
    __shared__ uint32_t s_tile[2];        // the tile staged in each buffer
    __shared__ TileInfo s_ti[NB];         // its position and field constants

    for (int j = threadIdx.x; j < 512; j += SCTA) smulti[j] = D.multi[j];
    if (threadIdx.x == 0) {
        s_err = 0;
        s_ncp = 0;
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        mbar_init_fence();
    }
    uint32_t tma_pending = 0, tma_phase = 0;  // per buffer: a TMA load in flight; the parity it completes
    uint32_t nvisits = 0;                     // CHECK_LIST: dirty vertices this warp visited
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float qnan = __int_as_float(0x7fc00000);

    // The tile's descriptors into buffer b with cp.async, one row of TX per
    // warp at a time.  The field's constants are read once, into registers:
    // each cp.async is an asm statement with a memory clobber, after which a
    // read through the field table would be issued again.
    auto stage_desc = [&](const int b, const TileGeo &G, const FieldDesc &F) {
        const uint32_t nx = F.nx, ny = F.ny, nz = F.nz;
        const uint32_t *const desc = D.desc + F.vbase;
        const uint32_t X = (uint32_t)G.x0 + lane;
        for (int row = warp; row < ROWS; row += STWARPS) {
            const uint32_t Y = (uint32_t)G.y0 + row % TY, Z = (uint32_t)G.z0 + row / TY;
            if (X < nx && Y < ny && Z < nz) cp_async4(&s_desc[b][row * TX + lane], desc + ((uint64_t)Z * ny + Y) * nx + X);
        }
    };

    // Stage tile into buffer b: the halo rows (one warp per row of HXP values,
    // x0-1 .. x0+TX) and, for CHECK_LIST, the tile's dirty row words.
    auto stage = [&](const uint32_t tile, const int b) {
        const uint32_t fid = field_of_tile(D, tile);
        const uint32_t tmab = D.fields[fid].tma;
        const bool tma_halo = (tmab & ((MODE == SM_SETUP || MODE == SM_CLASSIFY) ? TMA_SETUP : TMA_G)) != 0;
        const bool tma_desc = CHECK && (tmab & TMA_DESC) != 0;
        if (tma_halo) {  // the whole halo (NaN outside the field) in one TMA load per array
            tma_pending |= 1u << b;
            if (CHECK && !tma_desc)  // descriptors without a tensor map (rows not 16-byte multiples): cp.async
                stage_desc(b, tile_geo_of(D, tile, fid), D.fields[fid]);
            if (warp == 0) {  // warp 0 alone: the geometry, the dirty words and the TMA loads
                const TileGeo G = tile_geo_of(D, tile, fid);
                const FieldDesc &F = D.fields[fid];
                const uint32_t ny = F.ny, nz = F.nz;
                if (MODE == SM_CHECK_LIST && lane < ROWS) {
                    const uint32_t y = (uint32_t)G.y0 + lane % TY, z = (uint32_t)G.z0 + lane / TY;
                    if (y < ny && z < nz)
                        cp_async4(&s_rw[b][lane], D.dirty + F.wbase + ((uint64_t)z * ny + y) * F.tnx + G.tx);
                    else s_rw[b][lane] = 0;
                }
                if (lane == 0) {
                    s_ti[b] = tile_info(G, F);
                    const CUtensorMap *maps = D.tmaps + (uint64_t)TMAPS * G.fid;
                    fence_proxy_async();  // the buffer's earlier reads come first
                    mbar_expect_tx(&s_mbar[b], (MODE == SM_SETUP ? 2u : 1u) * (uint32_t)(HALO_N * sizeof(float)) +
                                                   (tma_desc ? (uint32_t)(TILE_V * sizeof(uint32_t)) : 0u));
                    tma_load_3d(sa[b], maps + ((MODE == SM_SETUP || MODE == SM_CLASSIFY) ? 0 : 2), G.x0 - XOFF,
                                G.y0 - 1, G.z0 - 1, &s_mbar[b]);
                    if (MODE == SM_SETUP) tma_load_3d(sb[b], maps + 1, G.x0 - XOFF, G.y0 - 1, G.z0 - 1, &s_mbar[b]);
                    if (tma_desc) tma_load_3d(s_desc[b], maps + 3, G.x0, G.y0, G.z0, &s_mbar[b]);
                }
            }
            return;
        }
        // fields without tensor maps: every thread copies its share with cp.async
        const TileGeo G = tile_geo_of(D, tile, fid);
        const FieldDesc &F = D.fields[fid];
        if (threadIdx.x == 0) s_ti[b] = tile_info(G, F);
        const uint32_t nx = F.nx, ny = F.ny, nz = F.nz;
        if (MODE == SM_CHECK_LIST && threadIdx.x < ROWS) {
            const uint32_t y = (uint32_t)G.y0 + threadIdx.x % TY, z = (uint32_t)G.z0 + threadIdx.x / TY;
            if (y < ny && z < nz) cp_async4(&s_rw[b][threadIdx.x], D.dirty + F.wbase + ((uint64_t)z * ny + y) * F.tnx + G.tx);
            else s_rw[b][threadIdx.x] = 0;
        }
        if (CHECK) stage_desc(b, G, F);
        const float *A = (MODE == SM_SETUP || MODE == SM_CLASSIFY) ? F.f : F.g;
        const float *B = F.fhat;
        const bool interior = G.x0 >= 1 && G.x0 + TX < (int)nx && G.y0 >= 1 && G.y0 + TY < (int)ny && G.z0 >= 1 &&
                              G.z0 + TZ < (int)nz;
        const bool aligned = ((reinterpret_cast<uintptr_t>(A) & 15u) == 0) &&
                             (MODE != SM_SETUP || (reinterpret_cast<uintptr_t>(B) & 15u) == 0);
        if (interior && aligned && (nx & 3u) == 0) {
            // every halo value is inside the field and each row's tile values
            // start on 16 bytes: 8 copies of 16 bytes per row plus its two ends
            const uint64_t nxy = (uint64_t)nx * ny;
            const uint64_t corner = ((uint64_t)(G.z0 - 1) * ny + (uint64_t)(G.y0 - 1)) * nx + G.x0;
            const float *base = A + corner;
            const float *base_b = B + corner;
            constexpr int PARTS = TX / 4 + 2;
            for (int j = threadIdx.x; j < HY * HZ * PARTS; j += SCTA) {
                const int row = j / PARTS, part = j - row * PARTS;
                const int hz = row / HY, hy = row - hz * HY;
                const uint64_t off = (uint64_t)hz * nxy + (uint64_t)hy * nx;
                const float *g = base + off;
                float *sr = sa[b] + row * HXP + XOFF;
                if (part < TX / 4) cp_async16(sr + 4 * part, g + 4 * part);
                else if (part == TX / 4) cp_async4(sr - 1, g - 1);
                else cp_async4(sr + TX, g + TX);
                if (MODE == SM_SETUP) {
                    const float *h = base_b + off;
                    float *tr = sb[b] + row * HXP + XOFF;
                    if (part < TX / 4) cp_async16(tr + 4 * part, h + 4 * part);
                    else if (part == TX / 4) cp_async4(tr - 1, h - 1);
                    else cp_async4(tr + TX, h + TX);
                }
            }
            return;
        }
        for (int row = warp; row < HY * HZ; row += STWARPS) {
            const int hz = row / HY, hy = row - hz * HY;
            const int Y = G.y0 - 1 + hy, Z = G.z0 - 1 + hz;
            const bool rin = Y >= 0 && Z >= 0 && Y < (int)ny && Z < (int)nz;
            const uint64_t rb = rin ? ((uint64_t)Z * ny + (uint64_t)Y) * nx : 0;
            const int X0 = G.x0 - 1 + lane, X1 = G.x0 + TX - 1 + lane;
            const bool in0 = rin && X0 >= 0 && X0 < (int)nx;
            const bool in1 = rin && lane < 2 && X1 < (int)nx;
            float *sr = sa[b] + row * HXP + (XOFF - 1);  // slot of x0 - 1
            if (in0) cp_async4(sr + lane, A + rb + X0);
            else sr[lane] = qnan;
            if (lane < 2) {
                if (in1) cp_async4(sr + TX + lane, A + rb + X1);
                else sr[TX + lane] = qnan;
            }
            if (MODE == SM_SETUP) {
                float *tr = sb[b] + row * HXP + (XOFF - 1);
                if (in0) cp_async4(tr + lane, B + rb + X0);
                else tr[lane] = qnan;
                if (lane < 2) {
                    if (in1) cp_async4(tr + TX + lane, B + rb + X1);
                    else tr[TX + lane] = qnan;
                }
            }
        }
    };

    // Check (or classify) the staged tile in buffer b; ends with a barrier.
    auto process = [&](const uint32_t tile, const int b) {
        const TileInfo &T = s_ti[b];
        const uint32_t fid = T.G.fid, tx = T.G.tx;
        const int x0 = T.G.x0, y0 = T.G.y0, z0 = T.G.z0;
        const uint32_t nx = T.nx, ny = T.ny, nz = T.nz, tnx = T.tnx;
        const uint64_t vbase = T.vbase;
        const float *S = sa[b];
        const uint32_t *RW = s_rw[b];
        // CHECK_LIST: the tile's dirty vertices are listed in shared memory in
        // row order (warp w lists the four rows of z-slab w at the offset the
        // row counts before them give, each lane writing its own bits); after a
        // block barrier warp w checks the batches w, w + STWARPS, ... of 32.
        int nvisit = 0;
        if (MODE == SM_CHECK_LIST) {
            if (threadIdx.x < ROWS && RW[threadIdx.x]) {  // the dirty bits are taken: clear them
                const uint32_t y = (uint32_t)y0 + threadIdx.x % TY, z = (uint32_t)z0 + threadIdx.x / TY;
                D.dirty[T.wbase + ((uint64_t)z * ny + y) * tnx + tx] = 0;
            }
            const uint32_t rc = lane < ROWS ? __popc(RW[lane]) : 0u;
            uint32_t incl = rc;
#pragma unroll
            for (int o = 1; o < ROWS; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            nvisit = (int)__shfl_sync(0xffffffffu, incl, ROWS - 1);
#pragma unroll
            for (int r = 0; r < TY; r++) {
                const int row = warp * TY + r;
                const uint32_t w = RW[row];
                const uint32_t before = __shfl_sync(0xffffffffu, incl - rc, row);
                if ((w >> lane) & 1u) s_vis[before + __popc(w & lanemask_lt())] = (uint16_t)((row << 5) | lane);
            }
            if (warp == 0) nvisits += (uint32_t)nvisit;
            __syncthreads();
        }
        const EmitGeo EG{nx, ny, tnx, T.tny, T.N, vbase, T.wbase, T.tbase};
        // index of the tile's first vertex (x0, y0, z0) in the field
        const uint64_t nxy = (uint64_t)nx * ny;
        const uint64_t tfirst = ((uint64_t)z0 * ny + (uint64_t)y0) * nx + (uint64_t)x0;
        const bool interior = x0 >= 1 && x0 + TX < (int)nx && y0 >= 1 && y0 + TY < (int)ny && z0 >= 1 &&
                              z0 + TZ < (int)nz;
        // vertices of this tile to visit: the batches of the dirty list
        // (CHECK_LIST) or all rows, warp w taking the rows of z-slab w
        const int vend = MODE == SM_CHECK_LIST ? nvisit : (warp + 1) * TY * TX;
        for (int base = (MODE == SM_CHECK_LIST ? warp * 32 : warp * TY * TX); base < vend;
             base += (MODE == SM_CHECK_LIST ? STWARPS * 32 : TX)) {
            int lx, ly, lz;
            bool sel = true;
            if (MODE == SM_CHECK_LIST) {
                const int k = base + lane;
                sel = k < nvisit;
                const uint32_t code = sel ? s_vis[k] : 0u;
                lx = (int)(code & 31u);
                ly = (int)((code >> 5) % TY);
                lz = (int)((code >> 5) / TY);
            } else {
                const int rr = base / TX;
                lx = lane;
                ly = rr % TY;
                lz = rr / TY;
            }
            const uint32_t x = (uint32_t)(x0 + lx), y = (uint32_t)(y0 + ly), z = (uint32_t)(z0 + lz);
            const bool in = sel && (interior || (x < nx && y < ny && z < nz));
            const int c = ((lz + 1) * HY + (ly + 1)) * HXP + (lx + XOFF);
            bool cp = false, listed = false;
            uint32_t req = 0;
            const uint64_t i = tfirst + (uint64_t)lz * nxy + (uint64_t)ly * nx + (uint64_t)lx;
            // the vertex's neighbours in the field (all 14 away from the boundary)
            const uint32_t valid = interior ? 0x3FFFu : valid_slots(x, y, z, nx, ny, nz);
            if (in) {
                if (MODE == SM_SETUP || MODE == SM_CLASSIFY) {
                    Stn sf = stencil15(S, c);
                    sf.valid = valid;
                    const uint32_t L = sf.mask, U = sf.valid & ~sf.mask;
                    const bool mn = L == 0, mxx = !mn && U == 0;
                    const bool join = !mn && !mxx && multi_bit(smulti, L);
                    const bool split = !mn && !mxx && multi_bit(smulti, U);
                    cp = mn || mxx || join || split;
                    listed = (MODE == SM_SETUP && D.events) ? (join || split) : cp;
                    const uint32_t d = sf.up | (sf.dn << 4) | (sf.mask << 8) |
                                       ((join || split) ? D_SADDLE : 0u) | (listed ? D_CP : 0u);
                    if (MODE == SM_CLASSIFY) {
                        desc_out[i] = d;
                        if (type_out)
                            type_out[i] = (uint8_t)(mn ? 1 : (mxx ? 2 : ((join ? 4 : 0) | (split ? 8 : 0))));
                    } else {
                        const float *SB = sb[b];
                        const float fv = S[c], hv = SB[c];
                        uint32_t e = 0;
                        if (!isfinite(fv) || !isfinite(hv)) e = ERR_NONFINITE;
                        else if (hv < __fsub_rn(fv, T.xi) || hv > __fadd_rn(fv, T.xi)) e = ERR_BOUND;
                        if (e) atomicOr(&s_err, e);
                        D.desc[vbase + i] = d;  // edit count k = 0 in the top byte
                        if (T.gm) T.gm[((uint64_t)z * ny + y) * T.pitch + x] = hv;  // g is kept there
                        else T.g[i] = hv;
                        if (D.events && (mn || mxx)) D.cp_rank[vbase + i] = 0;  // no linked saddle yet
                        Stn sg = stencil15(SB, c);
                        sg.valid = valid;
                        req = request_mask(smulti, d, sg);
                    }
                } else {
                    const uint32_t d = s_desc[b][(lz * TY + ly) * TX + lx];
                    Stn sg = stencil15(S, c);
                    sg.valid = valid;
                    req = request_mask(smulti, d, sg);
                }
            }
            if (MODE != SM_CLASSIFY && req) emit_targets<MODE == SM_PINNED>(D, EG, x, y, z, req);
            if (MODE == SM_SETUP) {
                const uint32_t w = __ballot_sync(0xffffffffu, listed);
                if (lane == 0 && y < ny && z < nz)
                    D.cpwords[T.wbase + ((uint64_t)z * ny + y) * tnx + tx] = w;
                if (D.events) {
                    const uint32_t c = __popc(__ballot_sync(0xffffffffu, cp));
                    if (lane == 0 && c) atomicAdd(&s_ncp, c);
                }
            }
        }
        if (MODE == SM_SETUP || MODE == SM_CLASSIFY) __syncthreads();  // the block's error and CP counts
        if (MODE == SM_SETUP && threadIdx.x == 0 && s_err) {
            atomicOr(&D.fst[fid].err, s_err);
            s_err = 0;
        }
        if (MODE == SM_SETUP && threadIdx.x == 0 && s_ncp) {
            atomicAdd(&D.fst[fid].ncp_all, (unsigned long long)s_ncp);
            s_ncp = 0;
        }
        if (MODE == SM_CLASSIFY) __syncthreads();
    };

    // Tile source, advanced by warp 0; its state lives in shared memory so that
    // it holds no registers while tiles are checked.
    struct Source {
        unsigned long long it, it1, its, ntiles;  // ranges and pinned lists; tiles taken
        const uint32_t *plist;
        uint32_t fi;
        uint32_t nxt, end, step, pend, pbase;  // CHECK_LIST: next position, taken flags of the last probe
    };
    __shared__ Source src;
    if (threadIdx.x == 0) {
        src.it = src.it1 = src.ntiles = 0;
        src.its = 1;
        src.plist = nullptr;
        src.fi = src.nxt = src.end = src.pend = src.pbase = 0;
        src.step = 1;
        if (MODE == SM_CHECK_LIST) {
            work_range(D, D.total_tiles, blockIdx.x, gridDim.x, src.nxt, src.end, src.step);
        } else if (MODE != SM_PINNED) {
            tile_range(D, t1 - t0, src.it, src.it1, src.its);
        }
    }
    __syncthreads();
    auto next_tile = [&]() -> uint32_t {  // warp 0, all lanes
        uint32_t t = NO_TILE;
        if (MODE == SM_CHECK_LIST) {
            uint32_t nxt = src.nxt, pend = src.pend, pbase = src.pbase;
            const uint32_t end = src.end, step = src.step;
            uint32_t taken = 0;
            while (pend == 0 && nxt < end) {
                // probe the next 32 tiles of this block at once; take the flagged ones
                const uint64_t ti = (uint64_t)nxt + (uint64_t)lane * step;
                const bool f = ti < end && D.tile_flag[ti] != 0;
                if (f) D.tile_flag[ti] = 0;
                pend = __ballot_sync(0xffffffffu, f);
                pbase = nxt;
                taken += __popc(pend);
                const uint64_t nn = (uint64_t)nxt + 32ull * step;
                nxt = nn < end ? (uint32_t)nn : end;
            }
            if (pend) {
                t = pbase + (uint32_t)(__ffs(pend) - 1) * step;
                pend &= pend - 1;
            }
            __syncwarp();
            if (lane == 0) {
                src.nxt = nxt;
                src.pend = pend;
                src.pbase = pbase;
                src.ntiles += taken;
            }
        } else if (MODE == SM_PINNED) {
            unsigned long long it = src.it, it1 = src.it1, its = src.its;
            const uint32_t *plist = src.plist;
            uint32_t fi = src.fi;
            while (it >= it1 && fi < nf) {
                const unsigned long long count = D.fst[fids[fi]].pin_tile_count;
                plist = D.fields[fids[fi]].pin_tiles;
                fi++;
                tile_range(D, count, it, it1, its);
            }
            if (it < it1) {
                t = plist[it];
                it += its;
            }
            __syncwarp();
            if (lane == 0) {
                src.it = it;
                src.it1 = it1;
                src.its = its;
                src.plist = plist;
                src.fi = fi;
            }
        } else {
            const unsigned long long it = src.it;
            if (it < src.it1) {
                t = t0 + (uint32_t)it;
                __syncwarp();
                if (lane == 0) src.it = it + src.its;
            }
        }
        __syncwarp();
        return t;
    };

    if (warp == 0) {
        const uint32_t t = next_tile();
        if (lane == 0) s_tile[0] = t;
    }
    __syncthreads();
    {
        const uint32_t t = s_tile[0];
        if (t != NO_TILE) stage(t, 0);
        cp_async_commit();
    }
    for (int b = 0;; b ^= 1) {
        const uint32_t cur = s_tile[b];
        if (cur == NO_TILE) break;
        if (warp == 0) {
            const uint32_t t = next_tile();
            if (lane == 0) s_tile[b ^ 1] = t;
        }
        cp_async_wait_all();  // this thread's copies of `cur`, the only ones in flight, have landed
        bool ok = true;
        if (tma_pending & (1u << b)) {  // and the tile's TMA load
            ok = mbar_wait(&s_mbar[b], (tma_phase >> b) & 1u);
            tma_phase ^= 1u << b;
            tma_pending &= ~(1u << b);
        }
        // everyone's have landed; s_tile[b ^ 1] is set; buffer b ^ 1 is free
        if (__syncthreads_or(!ok)) {  // a load that never completed: report, give it one more bounded wait, stop
            if (threadIdx.x == 0) atomicOr(&D.ls->fault, 1u);
            if (!ok) mbar_wait(&s_mbar[b], ((tma_phase >> b) & 1u) ^ 1u);
            break;
        }
        const uint32_t nxt = s_tile[b ^ 1];
        if (nxt != NO_TILE) stage(nxt, b ^ 1);  // lands while `cur` is checked
        cp_async_commit();
        process(cur, b);
    }
    if (MODE == SM_CHECK_LIST && threadIdx.x == 0 && src.ntiles) atomicAdd(&D.ls->sum_tiles, src.ntiles);
    if (MODE == SM_CHECK_LIST && lane == 0 && nvisits) atomicAdd(&D.ls->sum_visits, (unsigned long long)nvisits);
}

template <int MODE>
__global__ void __launch_bounds__(SCTA, MODE == SM_SETUP ? 8 : ((MODE == SM_CHECK_LIST || MODE == SM_PINNED) ? 10 : 12))
    k_stencil(Dev D, uint32_t *desc_out, uint8_t *type_out, uint32_t t0, uint32_t t1, const uint32_t *fids, uint32_t nf)
{
    stencil_tiles<MODE>(D, desc_out, type_out, t0, t1, fids, nf);
}

// ------------------------------------------------------------ block scan helpers
// Exclusive scan of one uint32 per thread across a block of NT threads;
// returns the block total.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan_n(uint32_t v, uint32_t &excl, uint32_t *swarp)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) swarp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? swarp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) swarp[lane] = w;
    }
    __syncthreads();
    const uint32_t before = warp ? swarp[warp - 1] : 0;
    const uint32_t total = swarp[NW - 1];
    excl = before + x - v;
    __syncthreads();
    return total;
}

// Exclusive scan of n uint32 values into uint64 offsets, *total = the sum
// (if not null).  One block of SCAN_NT threads walks the input in tiles of
// 4 * SCAN_NT values (each thread one uint4 where the input allows it), so that
// every load and store is coalesced; a running carry joins the tiles.
__global__ void __launch_bounds__(SCAN_NT) k_scan_u32(const uint32_t *in, unsigned long long *out, uint64_t n,
                                                      unsigned long long *total)
{
    static_assert(SCAN_NT == 32 * 32, "two-level warp scan: 32 warps of 32 lanes");
    __shared__ unsigned long long sw[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const bool vec = (reinterpret_cast<uintptr_t>(in) & 15u) == 0;
    for (uint64_t base = 0; base < n; base += 4 * SCAN_NT) {
        const uint64_t j = base + 4ull * threadIdx.x;
        uint32_t v[4];
        if (vec && j + 3 < n) {
            const uint4 w = *reinterpret_cast<const uint4 *>(in + j);
            v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = (j + u < n) ? in[j + u] : 0u;
        }
        const unsigned long long tsum = (unsigned long long)v[0] + v[1] + v[2] + v[3];
        unsigned long long x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sw[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = sw[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            sw[lane] = w;
        }
        __syncthreads();
        unsigned long long run = s_carry + (warp ? sw[warp - 1] : 0ull) + x - tsum;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (j + u < n) out[j + u] = run;
            run += v[u];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += sw[31];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = s_carry;
}

// In-place exclusive scan of n uint32 values (sum < 2^32); one block of 1024
// threads walks the array in tiles of 4096 (each thread one uint4), so every
// load and store is coalesced.
__global__ void __launch_bounds__(SCAN_NT) k_scan_inplace_u32(uint32_t *a, uint64_t n)
{
    static_assert(SCAN_NT == 32 * 32, "two-level warp scan: 32 warps of 32 lanes");
    __shared__ uint32_t sw[32];
    __shared__ uint32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < n; base += 4 * SCAN_NT) {
        const uint64_t j = base + 4ull * threadIdx.x;
        uint32_t v[4];
        if (j + 3 < n) {
            const uint4 w = *reinterpret_cast<const uint4 *>(a + j);
            v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = (j + u < n) ? a[j + u] : 0u;
        }
        const uint32_t tsum = v[0] + v[1] + v[2] + v[3];
        uint32_t x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sw[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = sw[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            sw[lane] = w;
        }
        __syncthreads();
        uint32_t run = s_carry + (warp ? sw[warp - 1] : 0u) + x - tsum;
        uint32_t out[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            out[u] = run;
            run += v[u];
        }
        if (j + 3 < n) {
            *reinterpret_cast<uint4 *>(a + j) = make_uint4(out[0], out[1], out[2], out[3]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (j + u < n) a[j + u] = out[u];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += sw[31];
        __syncthreads();
    }
}

// ------------------------------------------------------------ CP compaction
constexpr int WPT = WBLOCK / CTA;  // cp-bitmap words per thread

__device__ __forceinline__ uint32_t field_of_word(const Dev &D, uint64_t w, uint32_t lo, uint32_t hi)
{
    hi -= 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (D.fields[mid].wbase <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(CTA) k_cp_count(Dev D, uint64_t wblk0)
{
    __shared__ uint32_t sw[WARPS];
    const uint64_t w0 = (wblk0 + blockIdx.x) * WBLOCK + threadIdx.x * WPT;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < WPT; j++) c += __popc(D.cpwords[w0 + j]);
    uint32_t ex;
    uint32_t tot = block_excl_scan_n<CTA>(c, ex, sw);
    if (threadIdx.x == 0) D.blk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(CTA) k_cp_write(Dev D, SetupRange R)
{
    const uint64_t wblk0 = R.wblk0, cp0 = R.cp0;
    __shared__ uint32_t sw[WARPS];
    const uint64_t blk0 = (wblk0 + blockIdx.x) * WBLOCK;
    const uint32_t fid = field_of_word(D, blk0, R.fid0, R.fid1);
    const FieldDesc &F = D.fields[fid];
    const uint64_t w0 = blk0 + threadIdx.x * WPT;
    uint32_t words[WPT];
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < WPT; j++) {
        words[j] = D.cpwords[w0 + j];
        c += __popc(words[j]);
    }
    uint32_t ex;
    block_excl_scan_n<CTA>(c, ex, sw);
    unsigned long long pos = cp0 + D.blk_off[blockIdx.x] + ex;
    if (blk0 == F.wbase && threadIdx.x == 0) D.fst[fid].cp_base = cp0 + D.blk_off[blockIdx.x];
    const uint64_t ny = F.ny;
#pragma unroll
    for (int j = 0; j < WPT; j++) {
        uint32_t w = words[j];
        if (!w) continue;
        const uint64_t wl = w0 + j - F.wbase;
        const uint64_t row = wl / F.tnx, wx = wl % F.tnx;
        const uint64_t y = row % ny, z = row / ny;
        while (w) {
            const int b = __ffs(w) - 1;
            w &= w - 1;
            const uint64_t x = wx * 32 + b;
            const uint64_t t = x + (uint64_t)F.nx * (y + ny * z);
            D.cp_key[0][pos] = fkey(F.f[t]);
            D.cp_ent[0][pos] = ((unsigned long long)fid << LOCAL_BITS) | t;
            pos++;
        }
    }
}

__global__ void __launch_bounds__(SMALL_NT) k_cp_ncp(Dev D, SetupRange R)
{
    const unsigned long long end = R.cp0 + *R.cp_count;
    for (uint32_t f = R.fid0 + threadIdx.x + blockIdx.x * blockDim.x; f < R.fid1; f += blockDim.x * gridDim.x) {
        const unsigned long long b = D.fst[f].cp_base;
        const unsigned long long e = (f + 1 < R.fid1) ? D.fst[f + 1].cp_base : end;
        D.fst[f].ncp = e - b;
    }
}

// ------------------------------------------------------------ radix sort (stable LSD)
// The sort kernels run RADIX threads per block: thread d owns digit d.
constexpr int RADIX = 256;
constexpr int SWARPS = RADIX / 32;
// Pass p < 4: digit p of the 32-bit value key; pass p >= 4: digit p-4 of the field id.
__device__ __forceinline__ uint32_t sort_digit(int pass, uint32_t key, unsigned long long ent)
{
    if (pass < 4) return (key >> (8 * pass)) & 255u;
    return (uint32_t)(ent >> (LOCAL_BITS + 8 * (pass - 4))) & 255u;
}

__global__ void __launch_bounds__(RADIX) k_sort_hist(Dev D, int pass, const uint32_t *ksrc,
                                                     const unsigned long long *esrc, const unsigned long long *countp)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const unsigned long long count = *countp;
    const unsigned long long chunk = (count + gridDim.x - 1) / gridDim.x;
    const unsigned long long b = blockIdx.x * chunk, e = min(count, b + chunk);
    for (unsigned long long j = b + threadIdx.x; j < e; j += RADIX) {
        const uint32_t key = pass < 4 ? ksrc[j] : 0u;
        const unsigned long long ent = pass < 4 ? 0ull : esrc[j];
        atomicAdd(&h[sort_digit(pass, key, ent)], 1u);
    }
    __syncthreads();
    D.hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// One LSD pass, tile by tile: each block owns a contiguous chunk of the input
// (the same chunk its histogram counted) and takes it SORT_TILE elements at a
// time.  Warp w ranks the w-th 384-element slice of the tile by itself, 32
// elements per round (warp match for the rank within a round, a running count
// per digit in the warp's shared counters); then the warps' counts are
// prefixed per digit and the digits' tile counts scanned, which places every
// element of the tile in digit order, stably, in shared memory; from there
// consecutive threads write consecutive positions of each digit's run.
// last != 0: this is the final pass; also record each critical point's rank
// within its field (cp_rank), which the frontier uses to find its CP pairs,
// and its value in sorted order (gs).
constexpr int SORT_ROUNDS = 12;
constexpr int SORT_TILE = RADIX * SORT_ROUNDS;

__global__ void __launch_bounds__(RADIX) k_sort_scatter(Dev D, int pass, const uint32_t *ksrc,
                                                        const unsigned long long *esrc, uint32_t *kdst,
                                                        unsigned long long *edst, int last,
                                                        const unsigned long long *countp, uint64_t cp0)
{
    __shared__ uint32_t s_key[SORT_TILE];
    __shared__ unsigned long long s_ent[SORT_TILE];
    __shared__ uint32_t s_wc[SWARPS][RADIX];  // a warp's running digit counts, then their prefixes
    __shared__ uint32_t s_tbase[RADIX];       // first position of each digit in the tile
    __shared__ uint32_t s_gbase[RADIX];       // next output position of each digit for this block
    __shared__ uint32_t s_sw[SWARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long count = *countp;
    const unsigned long long chunk = (count + gridDim.x - 1) / gridDim.x;
    const unsigned long long b = blockIdx.x * chunk, e = min(count, b + chunk);
    const bool move_keys = pass < 3;  // keys are not needed after the last value pass
    s_gbase[threadIdx.x] = D.hist[threadIdx.x * gridDim.x + blockIdx.x];
    uint32_t *wc = s_wc[warp];
    for (unsigned long long base = b; base < e; base += SORT_TILE) {
        const uint32_t ntile = (uint32_t)min((unsigned long long)SORT_TILE, e - base);
        const uint32_t w0 = (uint32_t)warp * (SORT_TILE / SWARPS);  // this warp's slice of the tile
        uint32_t key[SORT_ROUNDS], dig[SORT_ROUNDS], lrank[SORT_ROUNDS];
        unsigned long long ent[SORT_ROUNDS];
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; r++) {  // all loads of the slice first
            const uint32_t jt = w0 + (uint32_t)r * 32 + lane;
            key[r] = 0;
            ent[r] = 0;
            if (jt < ntile) {
                if (pass < 4) key[r] = ksrc[base + jt];
                ent[r] = esrc[base + jt];
            }
        }
#pragma unroll
        for (int j = 0; j < RADIX / 32; j++) wc[j * 32 + lane] = 0;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; r++) {
            const bool valid = w0 + (uint32_t)r * 32 + lane < ntile;
            dig[r] = valid ? sort_digit(pass, key[r], ent[r]) : 0x100u;  // 0x100: never a real digit
            const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
            const uint32_t rank = __popc(peers & lanemask_lt());
            const uint32_t before = valid ? wc[dig[r]] : 0u;
            __syncwarp();
            if (valid && rank == 0) wc[dig[r]] = before + __popc(peers);
            __syncwarp();
            lrank[r] = before + rank;
        }
        __syncthreads();
        // per digit: prefix of the warps' counts, and the tile count
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < SWARPS; w++) {
            const uint32_t t = s_wc[w][threadIdx.x];
            s_wc[w][threadIdx.x] = run;
            run += t;
        }
        uint32_t ex;
        block_excl_scan_n<RADIX>(run, ex, s_sw);  // (has barriers)
        s_tbase[threadIdx.x] = ex;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; r++) {
            if (dig[r] < 0x100u) {
                const uint32_t p = s_tbase[dig[r]] + wc[dig[r]] + lrank[r];
                s_key[p] = key[r];
                s_ent[p] = ent[r];
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < ntile; i += RADIX) {
            const uint32_t k = s_key[i];
            const unsigned long long en = s_ent[i];
            const uint32_t d = sort_digit(pass, k, en);
            const uint32_t pos = s_gbase[d] + (i - s_tbase[d]);
            if (move_keys) kdst[pos] = k;
            edst[pos] = en;
            if (last) {
                const uint32_t fid = (uint32_t)(en >> LOCAL_BITS);
                const FieldDesc &F = D.fields[fid];
                D.cp_rank[F.vbase + (en & LOCAL_MASK)] = (uint32_t)(cp0 + pos - D.fst[fid].cp_base);
                D.gs[cp0 + pos] = F.fhat[en & LOCAL_MASK];  // g == f_hat before the first edit
            }
        }
        __syncthreads();
        s_gbase[threadIdx.x] += run;
    }
}

// ------------------------------------------------------------ pair check (Sec. 4.3)
enum { PM_ALL = 0, PM_LIST = 1, PM_PINNED = 2 };

// Merge and split event constraint (Sec. 4.2, C3) at listed saddle q:
// Extremum Graph Pairing selects, among the extrema linked to q in f, the
// largest minimum and the smallest maximum (ties by index).  Where the
// selection under g differs, the join side requests the g-selection and the
// split side the f-selection, the lower of the two in f either way.  Writes the
// tiles of the requests (pinned targets only with PINNED_ONLY); returns their
// number.
template <bool PINNED_ONLY>
__device__ __forceinline__ int check_events(const Dev &D, unsigned long long q, uint32_t *tiles)
{
    const uint32_t c = D.ev_cnt[q];
    if (!c) return 0;
    const unsigned long long ent = D.o[q];
    const FieldDesc &F = D.fields[ent >> LOCAL_BITS];
    // g of vertex e: in the padded copy (row stride pitch) when the field has one
    const float *gp = F.gm ? F.gm : F.g;
    const uint32_t gpad = F.gm ? F.pitch - F.nx : 0u;
    auto g = [&](const uint32_t e) { return gp[(uint64_t)e + (uint64_t)(e / F.nx) * gpad]; };
    const uint32_t *lm = D.ev_list + D.ev_start[q];
    const uint32_t nm = c & 255u, nx = c >> 8;
    uint32_t target[2];
    int ntar = 0;
    if (nm) {
        const uint32_t *l = lm;
        const uint32_t sel = l[0];
        uint32_t best = sel;
        float bg = g(sel);
        for (uint32_t j = 1; j < nm; j++) {
            const uint32_t e = l[j];
            const float ge = g(e);
            if (bg < ge || (bg == ge && best < e)) {
                best = e;
                bg = ge;
            }
        }
        if (best != sel) target[ntar++] = best;
    }
    if (nx) {
        const uint32_t *l = lm + nm;
        const uint32_t sel = l[0];
        uint32_t best = sel;
        float bg = g(sel);
        for (uint32_t j = 1; j < nx; j++) {
            const uint32_t e = l[j];
            const float ge = g(e);
            if (ge < bg || (ge == bg && e < best)) {
                best = e;
                bg = ge;
            }
        }
        if (best != sel) target[ntar++] = sel;
    }
    int nt = 0;
    for (int k = 0; k < ntar; k++) {
        if (PINNED_ONLY && (D.desc[F.vbase + target[k]] >> D_K_SHIFT) <= F.N) continue;
        tiles[nt++] = request_vertex(D, F, target[k]);
    }
    return nt;
}

// Rule R3 on adjacent pairs (q, q+1) of the sorted critical points, reading
// their current values from gs (kept in sorted order by the apply kernel); the
// sorted entries are gathered only to resolve a tie by index or to name the
// target.  ALL: every pair of the CP segment [cp0, cp0 + *countp) (the first
// pass; pairs may straddle two fields).  LIST: the pairs whose bit the apply
// kernel set in pairbits (always inside one field); each warp scans whole
// words, takes and clears them, and each lane checks the pair of its bit.
// PINNED: the pinned-pair lists of fields fids[0..nf), pinned targets only.
// Under the original event constraints the listed points are the saddles
// (the pairs are rule C2) and each mode also evaluates rule C3 at saddles:
// ALL at every listed saddle, LIST at those whose event bit (set by the apply
// kernel when a linked extremum changed) is set, PINNED at those whose pinned
// event bit (set when a linked extremum was pinned) is set.
// (The body of k_pairs and of the fused pass kernel's CP-pair phase; blocks of
// NT threads.)
template <int PM, int NT>
__device__ __forceinline__ void pairs_body(const Dev &D, uint64_t cp0, const unsigned long long *countp,
                                           const uint32_t *fids, uint32_t nf)
{
    const int lane = threadIdx.x & 31;
    // evaluate pair q; true (and the tile of the request) when its target is requested
    auto check = [&](const unsigned long long q, uint32_t &tile) -> bool {
        const float ga = D.gs[q], gb = D.gs[q + 1];
        bool viol = gb < ga;
        unsigned long long a = 0;
        if (PM == PM_ALL || gb == ga) {
            a = D.o[q];
            const unsigned long long b = D.o[q + 1];
            if ((a >> LOCAL_BITS) != (b >> LOCAL_BITS)) viol = false;  // different fields
            else if (gb == ga) viol = (b & LOCAL_MASK) < (a & LOCAL_MASK);
        } else if (viol) {
            a = D.o[q];
        }
        if (!viol) return false;
        const FieldDesc &F = D.fields[a >> LOCAL_BITS];
        const uint64_t t = a & LOCAL_MASK;
        if (PM == PM_PINNED && (D.desc[F.vbase + t] >> D_K_SHIFT) <= F.N) return false;
        tile = request_vertex(D, F, t);
        return true;
    };
    const unsigned long long stride = (unsigned long long)gridDim.x * NT;
    const unsigned long long pw = (D.cp_cap + 31) / 32;  // pair-bit words; event bits, pinned event bits follow
    if (PM == PM_LIST || (PM == PM_PINNED && D.events)) {
        // each warp takes 32 consecutive words of pairbits at a time (one per
        // lane), clears them, numbers their set bits and checks them 32 at once.
        // LIST: the pair and event bits; PINNED: the event bits of saddles
        // linked to pinned extrema.
        const unsigned long long w0 = PM == PM_LIST ? 0ull : 2 * pw;
        const unsigned long long w1 = PM == PM_LIST ? (D.events ? 2 * pw : pw) : 3 * pw;
        const unsigned long long gw = ((unsigned long long)blockIdx.x * NT + threadIdx.x) >> 5;
        const unsigned long long nw = stride >> 5;
        uint32_t npairs = 0;
        for (unsigned long long c = gw; w0 + c * 32 < w1; c += nw) {
            const unsigned long long w = w0 + c * 32 + lane;
            const uint32_t word = w < w1 ? D.pairbits[w] : 0u;
            if (!__any_sync(0xffffffffu, word != 0)) continue;
            if (word) D.pairbits[w] = 0;  // taken
            const uint32_t cnt = __popc(word);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - cnt;
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            npairs += total;
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t k = base + lane;
                int src = 0;  // the last lane whose first number is <= k
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const uint32_t pe = __shfl_sync(0xffffffffu, excl, src + step);
                    if (pe <= k) src += step;
                }
                const uint32_t rword = __shfl_sync(0xffffffffu, word, src);
                const uint32_t rpre = __shfl_sync(0xffffffffu, excl, src);
                uint32_t tile = 0;
                if (k < total) {
                    const unsigned long long b = (w0 + c * 32 + src) * 32 + nth_set_bit(rword, (int)(k - rpre));
                    if (b < pw * 32) {
                        if (check(b, tile) && !D.apply_flag[tile]) D.apply_flag[tile] = 1;
                    } else {
                        uint32_t tl[2];
                        const unsigned long long q = b % (pw * 32);
                        const int nt = PM == PM_PINNED ? check_events<true>(D, q, tl) : check_events<false>(D, q, tl);
                        for (int u = 0; u < nt; u++)
                            if (!D.apply_flag[tl[u]]) D.apply_flag[tl[u]] = 1;
                    }
                }
            }
        }
        if (PM == PM_LIST) {
            if (lane == 0 && npairs) atomicAdd(&D.ls->sum_pairs, (unsigned long long)npairs);
            return;
        }
    }
    const uint32_t nouter = PM == PM_PINNED ? nf : 1u;
    for (uint32_t fi = 0; fi < nouter; fi++) {
        unsigned long long count;
        const uint32_t *list = nullptr;
        if (PM == PM_ALL) {
            const unsigned long long total = *countp;
            count = total ? total - 1 : 0;
        } else {
            count = D.fst[fids[fi]].pin_pair_count;
            list = D.fields[fids[fi]].pin_pairs;
        }
        for (unsigned long long j = (unsigned long long)blockIdx.x * NT + threadIdx.x; j < count; j += stride) {
            uint32_t tile = 0;
            if (check(list ? (unsigned long long)list[j] : cp0 + j, tile) && !D.apply_flag[tile])
                D.apply_flag[tile] = 1;
        }
    }
    if (PM == PM_ALL && D.events) {  // rule C3 at every listed saddle
        const unsigned long long count = *countp;
        for (unsigned long long j = (unsigned long long)blockIdx.x * NT + threadIdx.x; j < count; j += stride) {
            uint32_t tl[2];
            const int nt = check_events<false>(D, cp0 + j, tl);
            for (int u = 0; u < nt; u++)
                if (!D.apply_flag[tl[u]]) D.apply_flag[tl[u]] = 1;
        }
    }
}

template <int PM>
__global__ void __launch_bounds__(CTA) k_pairs(Dev D, uint64_t cp0, const unsigned long long *countp,
                                               const uint32_t *fids, uint32_t nf)
{
    pairs_body<PM, CTA>(D, cp0, countp, fids, nf);
}

// ------------------------------------------------------------ apply (Sec. 3.3)
// Exclusive warp prefix of c; one atomicAdd per warp reserves the slots.
// All 32 lanes must call it.
__device__ __forceinline__ unsigned long long warp_reserve(uint32_t c, unsigned long long *counter)
{
    const int lane = threadIdx.x & 31;
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + (x - c);
}

// The tiles holding the closed star of vertex (x, y, z), as a 27-bit mask of
// neighbour tiles (bit (ox+1) + 3 (oy+1) + 9 (oz+1); bit 13 = the vertex's own
// tile): the star's negative offsets are the non-zero vectors of {0,-1}^3 and
// its positive ones those of {0,1}^3, so on each side the other tiles it
// reaches are the non-zero combinations of the tile faces the vertex lies on.
__device__ __forceinline__ uint32_t star_tiles(uint32_t x, uint32_t y, uint32_t z, uint32_t nx, uint32_t ny,
                                               uint32_t nz)
{
    const uint32_t lo = ((x % TX) == 0 && x > 0 ? 1u : 0u) | ((y % TY) == 0 && y > 0 ? 2u : 0u) |
                        ((z % TZ) == 0 && z > 0 ? 4u : 0u);
    const uint32_t hi = ((x % TX) == TX - 1 && x + 1 < nx ? 1u : 0u) | ((y % TY) == TY - 1 && y + 1 < ny ? 2u : 0u) |
                        ((z % TZ) == TZ - 1 && z + 1 < nz ? 4u : 0u);
    uint32_t nb = 1u << 13;
#pragma unroll 1
    for (uint32_t m = lo; m; m = (m - 1) & lo)
        nb |= 1u << (13 - (int)(m & 1u) - 3 * (int)((m >> 1) & 1u) - 9 * (int)((m >> 2) & 1u));
#pragma unroll 1
    for (uint32_t m = hi; m; m = (m - 1) & hi)
        nb |= 1u << (13 + (int)(m & 1u) + 3 * (int)((m >> 1) & 1u) + 9 * (int)((m >> 2) & 1u));
    return nb;
}

enum { AM_PLAIN = 0, AM_FRONTIER = 1, AM_COUNT = 2 };

// The bounded monotone edit (Sec. 3.3) of requested vertex t of field F with
// its loaded descriptor d, f value fv, g value g0 and CP rank rk: unless it is
// pinned at the lossless bound, g takes one more step fl(g - Delta), or the
// bound fl(f - xi) once the steps are used up or the step would pass it (at the
// iteration cap the request is counted instead).  Keeps the CP's value in
// sorted order and marks, under the original event constraints, the saddles of
// a changed extremum.  Returns whether the vertex changed; pinned: it reached
// the bound; has_lo / has_hi: its CP pairs (q - 1, q) / (q, q + 1) exist and
// are to be checked (FRONTIER, or pinned).
// gm, tm: the field's padded copy of g, which holds g during the passes when
// the field has one (null otherwise; held in a register by the caller: the
// field table could be reloaded after every store), and the vertex's index in it.
template <int AM>
__device__ __forceinline__ bool edit_vertex(const Dev &D, const FieldDesc &F, float *gm, FieldState *S, uint64_t t,
                                            uint64_t tm, uint32_t d, float fv, float g0, uint32_t rk, bool capped,
                                            uint32_t &ncap, bool &pinned, bool &has_lo, bool &has_hi,
                                            unsigned long long &q)
{
    const uint32_t N = F.N;
    uint32_t kk = d >> D_K_SHIFT;
    if (kk > N) return false;  // a pinned target stays as it is
    if (capped) {
        ncap++;
        return false;
    }
    const float fl = __fsub_rn(fv, F.xi);
    float gv;
    if (kk < N) {
        const float tt = __fsub_rn(g0, F.delta);
        if (tt < fl) {
            gv = fl;
            kk = N + 1;
        } else {
            gv = tt;
            kk = kk + 1;
        }
    } else {
        gv = fl;
        kk = N + 1;
    }
    if (gm) gm[tm] = gv;  // g is kept in the padded copy during the passes
    else F.g[t] = gv;
    D.desc[F.vbase + t] = (d & D_F_MASK) | (kk << D_K_SHIFT);
    pinned = kk == N + 1;
    if (D.events && (AM == AM_FRONTIER || pinned) && !(d & D_CP) && rk != 0 &&
        ((d & 15u) == 7u || ((d >> 4) & 15u) == 7u)) {
        // an extremum linked to saddles: their rule C3 is checked next pass,
        // and by the residual check if it is pinned
        const unsigned long long pw = (D.cp_cap + 31) / 32;
        const uint32_t deg = D.ev_radj[rk];
        for (uint32_t j = 0; j < deg; j++) {
            const uint32_t qq = D.ev_radj[rk + 1 + j];
            if (AM == AM_FRONTIER) atomicOr(&D.pairbits[pw + (qq >> 5)], 1u << (qq & 31));
            if (pinned) atomicOr(&D.pairbits[2 * pw + (qq >> 5)], 1u << (qq & 31));
        }
    }
    if (d & D_CP) {  // value in sorted order; pairs inside the field
        const unsigned long long r = rk;
        q = S->cp_base + r;
        D.gs[q] = gv;
        if (AM == AM_FRONTIER || pinned) {
            has_lo = r >= 1;
            has_hi = r + 1 < S->ncp;
        }
    }
    return true;
}

// One tile holding requested vertices per warp iteration (warps work
// independently): a warp probes 32 of its tiles' flags at once, takes (and
// clears) the flagged ones and works through them.  The tile's 16 request words are read (and
// cleared) by lanes 0-15, the
// requested vertices are numbered by a warp prefix sum and worked through 32
// at a time, and the changed vertices are collected as row bits in the warp's
// shared words.
//   PLAIN / FRONTIER: apply the bounded edit (Sec. 3.3) to each requested,
//     unpinned vertex (at the iteration cap: count it instead), keep the CP
//     values in gs, queue CP pairs and pinned neighbourhoods; FRONTIER also
//     sets the next pass's dirty bits (the closed stars of the changed
//     vertices) and queues their tiles.
//   COUNT: add the requested (pinned) vertices to the field's residual.
// (The body of k_apply_tiles and of the fused pass kernel's apply phase; NW
// warps per block.  The tile flags and request words are read through L2: in
// the fused kernel other blocks wrote them earlier in the same launch.)
template <int AM, int NW>
__device__ __forceinline__ void apply_tiles(const Dev &D)
{
    __shared__ uint32_t s_cw_all[NW][ROWS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *s_cw = s_cw_all[warp];
    unsigned long long nreq = 0;
    uint32_t pb, pe, pst;
    work_range(D, D.total_tiles, blockIdx.x * NW + warp, gridDim.x * NW, pb, pe, pst);
    // The warp's flagged tiles, one at a time: probe 32 flags at once and take
    // the flagged ones.
    uint64_t p = pb;
    uint64_t pbase = 0;
    uint32_t pend = 0;
    auto next_tile = [&]() -> uint32_t {
        while (!pend && p < pe) {
            const uint64_t ti = p + (uint64_t)lane * pst;
            const bool flagged = ti < pe && __ldcg(&D.apply_flag[ti]) != 0;
            if (flagged) D.apply_flag[ti] = 0;
            pend = __ballot_sync(0xffffffffu, flagged);
            pbase = p;
            p += 32ull * pst;
        }
        if (!pend) return NO_TILE;
        const uint32_t t = (uint32_t)(pbase + (uint64_t)(__ffs(pend) - 1) * pst);
        pend &= pend - 1;
        return t;
    };
    for (uint32_t tile = next_tile(); tile != NO_TILE; tile = next_tile()) {
        const uint32_t fid = field_of_tile(D, tile);
        const FieldDesc &F = D.fields[fid];
        FieldState *S = &D.fst[fid];
        const uint32_t nx = F.nx, ny = F.ny, nz = F.nz, tnx = F.tnx, tny = F.tny;
        const uint32_t lt = (uint32_t)(tile - F.tbase);
        const uint32_t rest = fdiv(lt, F.div_tnx), tx = lt - rest * tnx;
        const uint32_t tz = fdiv(rest, F.div_tny), ty = rest - tz * tny;
        const uint32_t x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
        const uint64_t vbase = F.vbase, wbase = F.wbase;
        float *const gm = F.gm;
        const uint32_t pitch = F.pitch;
        uint32_t W = 0;  // lane r < ROWS: request word of tile row r (taken: read and cleared)
        if (lane < ROWS) {
            const uint32_t y = y0 + lane % TY, z = z0 + lane / TY;
            if (y < ny && z < nz) {
                uint32_t *wp = D.reqw + wbase + ((uint64_t)z * ny + y) * tnx + tx;
                W = __ldcg(wp);
                if (W) *wp = 0;
            }
            s_cw[lane] = 0;
        }
        const uint32_t c = __popc(W);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - c;  // requested vertices in the rows before this lane's row
        const int nvisit = (int)__shfl_sync(0xffffffffu, incl, ROWS - 1);
        nreq += (unsigned long long)nvisit;
        if (AM == AM_COUNT) {
            if (lane == 0 && nvisit) atomicAdd(&S->pinned_res, (unsigned long long)nvisit);
            continue;
        }
        __syncwarp();
        const bool err = S->err != 0, capped = S->iterations >= F.max_iters;
        uint32_t ncap = 0, pin_nb = 0;
        // After the edit of one vertex (lane-local results): queue its CP pairs
        // (FRONTIER), list the pairs and tiles around it if it was pinned.  All
        // lanes call it.
        auto after_edit = [&](const bool pinned, const bool has_lo, const bool has_hi, const unsigned long long q,
                              const uint32_t x, const uint32_t y, const uint32_t z) {
            if (AM == AM_FRONTIER) {  // the pairs (q, q+1) and (q-1, q) are checked next pass
                if (has_hi) atomicOr(&D.pairbits[q >> 5], 1u << (q & 31));
                if (has_lo) atomicOr(&D.pairbits[(q - 1) >> 5], 1u << ((q - 1) & 31));
            }
            const uint32_t npp = pinned ? (uint32_t)has_hi + (uint32_t)has_lo : 0u;
            if (__any_sync(0xffffffffu, npp != 0)) {
                const unsigned long long p = warp_reserve(npp, &S->pin_pair_count);
                if (pinned && has_hi) F.pin_pairs[p] = (uint32_t)q;
                if (pinned && has_lo) F.pin_pairs[p + (has_hi ? 1 : 0)] = (uint32_t)(q - 1);
            }
            if (pinned) pin_nb |= star_tiles(x, y, z, nx, ny, nz);
        };
        // the requested vertices, numbered by the row prefix sums, 32 at a time
        for (int base = 0; base < nvisit; base += 32) {
            const int k = base + lane;
            const bool sel = k < nvisit && !err;
            int row = 0;  // the last row whose first request number is <= k
#pragma unroll
            for (int step = ROWS / 2; step >= 1; step >>= 1) {
                const uint32_t pe = __shfl_sync(0xffffffffu, excl, row + step);
                if ((int)pe <= k) row += step;
            }
            const uint32_t rword = __shfl_sync(0xffffffffu, W, row);
            const uint32_t rpre = __shfl_sync(0xffffffffu, excl, row);
            bool pinned = false, has_lo = false, has_hi = false;
            unsigned long long q = 0;
            uint32_t x = 0, y = 0, z = 0;
            if (sel) {
                const int lx = nth_set_bit(rword, k - (int)rpre);
                x = x0 + lx;
                y = y0 + row % TY;
                z = z0 + row / TY;
                const uint64_t t = ((uint64_t)z * ny + y) * nx + x;
                // all loads of the vertex at once (f, g and the CP rank are not
                // needed for a pinned target or a regular vertex)
                const uint32_t d = D.desc[vbase + t];
                const uint64_t tm = ((uint64_t)z * ny + y) * pitch + x;  // index in the padded copy
                const float fv = F.f[t], g0 = gm ? gm[tm] : F.g[t];
                const uint32_t rk = D.cp_rank[vbase + t];
                if (edit_vertex<AM>(D, F, gm, S, t, tm, d, fv, g0, rk, capped, ncap, pinned, has_lo, has_hi, q))
                    atomicOr(&s_cw[row], 1u << lx);
            }
            after_edit(pinned, has_lo, has_hi, q, x, y, z);
        }
        // the residual check revisits the closed stars of pinned vertices: their
        // tiles are queued once per tile, one lane per neighbour tile
        pin_nb = __reduce_or_sync(0xffffffffu, pin_nb);
        if (pin_nb) {
            const int j = lane;
            const int ox = j % 3 - 1, oy = (j / 3) % 3 - 1, oz = j / 9 - 1;
            warp_mark_tiles(j < 27 && ((pin_nb >> j) & 1u),
                            (uint32_t)((int64_t)tile + ox + (int64_t)tnx * (oy + (int64_t)tny * oz)), D.pin_tile_bits,
                            F.pin_tiles, &S->pin_tile_count);
        }
        __syncwarp();
        const uint32_t cw = lane < ROWS ? s_cw[lane] : 0u;
        const bool any = __any_sync(0xffffffffu, cw != 0);
        ncap = __reduce_add_sync(0xffffffffu, ncap);
        if (lane == 0) {
            if (ncap) atomicAdd(&S->capped, (unsigned long long)ncap);
            if (any && !S->had_req) S->had_req = 1;
        }
        if (AM == AM_FRONTIER && any) {
            // dirty bits of the next pass: the closed stars of the changed
            // vertices.  Lane j gathers halo row j (of the 6 x 6 rows around the
            // tile) from the changed words of the tile rows whose star reaches
            // it: star row (dy, dz) of a changed word C covers C | C >> 1 for
            // the rows (0,0), (-1,0), (0,-1), (-1,-1) and C | C << 1 for (0,0),
            // (1,0), (0,1), (1,1); bits shifted out of the word go to the word
            // of the tile column on that side.  One atomic per word touched.
            uint32_t nb = 0;
            for (int j = lane; j < HY * HZ; j += 32) {
                const int hz = j / HY, hy = j - hz * HY;
                uint32_t m = 0, elo = 0, ehi = 0;
#pragma unroll
                for (int kk = 0; kk < 7; kk++) {
                    const int dy = (kk == 1 || kk == 3) ? -1 : ((kk == 4 || kk == 6) ? 1 : 0);
                    const int dz = (kk == 2 || kk == 3) ? -1 : ((kk == 5 || kk == 6) ? 1 : 0);
                    const int ly = hy - 1 - dy, lz = hz - 1 - dz;
                    if (ly < 0 || ly >= TY || lz < 0 || lz >= TZ) continue;
                    const uint32_t C = s_cw[lz * TY + ly];
                    m |= C;
                    if (kk <= 3) {
                        m |= C >> 1;
                        elo |= C & 1u;
                    }
                    if (kk == 0 || kk >= 4) {
                        m |= C << 1;
                        ehi |= C >> 31;
                    }
                }
                const int Y = (int)y0 - 1 + hy, Z = (int)z0 - 1 + hz;
                if (!(m | elo | ehi) || Y < 0 || Z < 0 || Y >= (int)ny || Z >= (int)nz) continue;
                const uint64_t wi = wbase + ((uint64_t)Z * ny + (uint64_t)Y) * tnx + tx;
                const int oy = hy == 0 ? -1 : (hy == TY + 1 ? 1 : 0);
                const int oz = hz == 0 ? -1 : (hz == TZ + 1 ? 1 : 0);
                if (m) {
                    atomicOr(&D.dirty[wi], m);
                    nb |= 1u << nb_index(0, oy, oz);
                }
                if (elo && tx > 0) {
                    atomicOr(&D.dirty[wi - 1], 0x80000000u);
                    nb |= 1u << nb_index(-1, oy, oz);
                }
                if (ehi && tx + 1 < tnx) {
                    atomicOr(&D.dirty[wi + 1], 1u);
                    nb |= 1u << nb_index(1, oy, oz);
                }
            }
            nb = __reduce_or_sync(0xffffffffu, nb);
            warp_mark_nb_tiles(nb, tile, tnx, tny, D.tile_flag);
        }
        __syncwarp();
    }
    if (AM != AM_COUNT && lane == 0 && nreq) atomicAdd(&D.ls->sum_requests, nreq);
}

template <int AM>
__global__ void __launch_bounds__(CTA, 4) k_apply_tiles(Dev D)
{
    apply_tiles<AM, WARPS>(D);
}

// ------------------------------------------------------------ event lists (set-up, Sec. 4.2)
// The extremum graph of f (Sec. 3.2 Step 1): a join saddle s is linked to the
// minimum where the steepest-descent path from any neighbour below s ends (split
// saddles: steepest ascent from the neighbours above, to maxima).  Path ends of
// all vertices come from pointer jumping on the steepest-neighbour links,
// E[v] <- E[E[v]] until nothing moves, both directions at once (E holds the
// descent links, E + total_v the ascent links, as arena indices).  It runs in
// place, since every value E[v] ever holds lies on v's path; bit 31 marks an
// entry that holds its path's end, which later rounds skip.
constexpr uint32_t EV_DONE = 0x80000000u;

// body(fid, F, t, x, y, z, in) for the vertices of the tiles taken by this
// block, one row of TX vertices per warp at a time (every thread calls it the
// same number of times; `in` is false outside the field).
template <class Body>
__device__ __forceinline__ void for_tile_vertices(const Dev &D, Body body)
{
    for (uint32_t tile = blockIdx.x; tile < D.total_tiles; tile += gridDim.x) {
        const uint32_t fid = field_of_tile(D, tile);
        const FieldDesc &F = D.fields[fid];
        const uint32_t lt = tile - (uint32_t)F.tbase;
        const uint32_t rest = fdiv(lt, F.div_tnx), tx = lt - rest * F.tnx;
        const uint32_t tz = fdiv(rest, F.div_tny), ty = rest - tz * F.tny;
        for (int j = threadIdx.x; j < TILE_V; j += CTA) {
            const uint32_t x = tx * TX + (uint32_t)(j % TX), y = ty * TY + (uint32_t)((j / TX) % TY);
            const uint32_t z = tz * TZ + (uint32_t)(j / (TX * TY));
            const bool in = x < F.nx && y < F.ny && z < F.nz;
            body(fid, F, in ? (uint32_t)(((uint64_t)z * F.ny + y) * F.nx + x) : 0u, x, y, z, in);
        }
    }
}

// Signed index offset of neighbour rank r in a field.
__device__ __forceinline__ int64_t rank_offset(const FieldDesc &F, int r)
{
    return (int64_t)rdx(r) + (int64_t)F.nx * ((int64_t)rdy(r) + (int64_t)F.ny * rdz(r));
}

// c slots from *counter for every thread of the block (all threads call it).
__device__ __forceinline__ unsigned long long block_reserve(uint32_t c, unsigned long long *counter, uint32_t *sw,
                                                            unsigned long long *sbase)
{
    uint32_t ex;
    const uint32_t total = block_excl_scan_n<CTA>(c, ex, sw);
    if (threadIdx.x == 0) *sbase = total ? atomicAdd(counter, (unsigned long long)total) : 0ull;
    __syncthreads();
    const unsigned long long b = *sbase;
    __syncthreads();
    return b + ex;
}

// E[v] = steepest-descent neighbour of v in f, E[total_v + v] = steepest
// ascent; an extremum links to itself, settled.  (Following the links inside
// each tile in shared memory first saves about one jump round on the bumps
// workload but costs as much as it saves.)
// Path ends inside a tile: each block takes whole tiles and follows the
// steepest links of their vertices in shared memory (synchronous pointer
// jumping, at most log2(TILE_V) rounds, since a path visits a vertex at most
// once), so that E starts at the first vertex of each path outside its tile,
// or at the path's extremum (settled); the global rounds then jump between
// tiles.  Both directions at once.
__global__ void __launch_bounds__(CTA) k_ev_init(Dev D, uint32_t *E)
{
    constexpr int PER = TILE_V / CTA;
    constexpr uint16_t OUT = 0xFFFFu;  // the link leaves the tile (or the vertex is settled)
    static_assert(TILE_V % CTA == 0 && TILE_V < OUT, "tile-local path slots");
    __shared__ uint16_t s_loc[2][TILE_V];  // next vertex inside the tile, or OUT
    __shared__ uint32_t s_end[2][TILE_V];  // with OUT: the arena value E takes
    for (uint32_t tile = blockIdx.x; tile < D.total_tiles; tile += gridDim.x) {
        const FieldDesc &F = D.fields[field_of_tile(D, tile)];
        const uint32_t lt = tile - (uint32_t)F.tbase;
        const uint32_t rest = fdiv(lt, F.div_tnx), tx = lt - rest * F.tnx;
        const uint32_t tz = fdiv(rest, F.div_tny), ty = rest - tz * F.tny;
        uint64_t av[PER];
        bool open = false;
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int j = threadIdx.x + q * CTA;
            const int lx = j % TX, ly = (j / TX) % TY, lz = j / (TX * TY);
            const uint32_t x = tx * TX + (uint32_t)lx, y = ty * TY + (uint32_t)ly, z = tz * TZ + (uint32_t)lz;
            av[q] = ~0ull;
            if (x >= F.nx || y >= F.ny || z >= F.nz) {  // no vertex here: no link points to it
                s_loc[0][j] = s_loc[1][j] = OUT;
                s_end[0][j] = s_end[1][j] = 0;
                continue;
            }
            const uint64_t a = F.vbase + ((uint64_t)z * F.ny + y) * F.nx + x;
            av[q] = a;
            const uint32_t d = D.desc[a];
#pragma unroll
            for (int side = 0; side < 2; side++) {
                const int r = side ? (int)(d & 15u) : (int)((d >> D_DN_SHIFT) & 15u);
                if (r == 7) {  // an extremum of this direction: its own end
                    s_loc[side][j] = OUT;
                    s_end[side][j] = (uint32_t)a | EV_DONE;
                    continue;
                }
                const int nx = lx + rdx(r), ny = ly + rdy(r), nz = lz + rdz(r);
                if (nx >= 0 && nx < TX && ny >= 0 && ny < TY && nz >= 0 && nz < TZ) {
                    s_loc[side][j] = (uint16_t)(nx + TX * (ny + TY * nz));
                    s_end[side][j] = 0;
                    open = true;
                } else {
                    s_loc[side][j] = OUT;
                    s_end[side][j] = (uint32_t)((int64_t)a + rank_offset(F, r));
                }
            }
        }
        // jump until every path has left the tile or ended (block-uniform test;
        // 10 rounds reach 2^10 > TILE_V steps, the bound only guards a corrupt descriptor)
        for (int round = 0; round < 12 && __syncthreads_or(open); round++) {
            uint16_t nl[PER][2];
            uint32_t ne[PER][2];
            open = false;
#pragma unroll
            for (int q = 0; q < PER; q++) {
                const int j = threadIdx.x + q * CTA;
#pragma unroll
                for (int side = 0; side < 2; side++) {
                    const uint16_t l = s_loc[side][j];
                    nl[q][side] = l == OUT ? OUT : s_loc[side][l];
                    ne[q][side] = l == OUT ? s_end[side][j] : s_end[side][l];
                    open |= nl[q][side] != OUT;
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < PER; q++) {
                const int j = threadIdx.x + q * CTA;
#pragma unroll
                for (int side = 0; side < 2; side++) {
                    s_loc[side][j] = nl[q][side];
                    s_end[side][j] = ne[q][side];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < PER; q++) {
            if (av[q] == ~0ull) continue;
            const int j = threadIdx.x + q * CTA;
            E[av[q]] = s_end[0][j];
            E[D.total_v + av[q]] = s_end[1][j];
        }
        __syncthreads();  // the next tile reuses the shared arrays
    }
}

// One jump round in both directions; sets ls->ev_changed if an entry changed.
// Tiles whose entries have all settled are marked in tdone and skipped.
__global__ void __launch_bounds__(CTA) k_ev_jump(Dev D, uint32_t *E, uint8_t *tdone)
{
    bool moved = false;
    for (uint32_t tile = blockIdx.x; tile < D.total_tiles; tile += gridDim.x) {
        if (tdone[tile]) continue;  // block-uniform
        const FieldDesc &F = D.fields[field_of_tile(D, tile)];
        const uint32_t lt = tile - (uint32_t)F.tbase;
        const uint32_t rest = fdiv(lt, F.div_tnx), tx = lt - rest * F.tnx;
        const uint32_t tz = fdiv(rest, F.div_tny), ty = rest - tz * F.tny;
        bool settled = true;
        for (int j = threadIdx.x; j < TILE_V; j += CTA) {
            const uint32_t x = tx * TX + (uint32_t)(j % TX), y = ty * TY + (uint32_t)((j / TX) % TY);
            const uint32_t z = tz * TZ + (uint32_t)(j / (TX * TY));
            if (x >= F.nx || y >= F.ny || z >= F.nz) continue;
            const uint64_t a = F.vbase + ((uint64_t)z * F.ny + y) * F.nx + x;
#pragma unroll
            for (int side = 0; side < 2; side++) {
                uint32_t *Es = E + (side ? D.total_v : 0ull);
                const uint32_t e = Es[a];
                if (e & EV_DONE) continue;
                const uint32_t e2 = Es[e];  // settled: the end of e's path, which is a's
                if (e2 != e) {
                    Es[a] = e2;
                    moved = true;
                }
                settled &= (e2 & EV_DONE) != 0;
            }
        }
        if (__syncthreads_and(settled) && threadIdx.x == 0) tdone[tile] = 1;
    }
    if (__syncthreads_or(moved) && threadIdx.x == 0) D.ls->ev_changed = 1;
}

// Neighbour slots whose offset has the given component (0: x, 1: y, 2: z) equal to v.
__host__ __device__ constexpr uint32_t slots_with(int comp, int v)
{
    uint32_t m = 0;
    for (int sl = 0; sl < 14; sl++) {
        const int r = rank_of(sl);
        const int c = comp == 0 ? rdx(r) : (comp == 1 ? rdy(r) : rdz(r));
        if (c == v) m |= 1u << sl;
    }
    return m;
}

// Neighbour slots of (x, y, z) inside the field.
__device__ __forceinline__ uint32_t valid_slots(const FieldDesc &F, uint32_t x, uint32_t y, uint32_t z)
{
    uint32_t m = 0x3FFFu;
    if (x == 0) m &= ~slots_with(0, -1);
    if (x + 1 == F.nx) m &= ~slots_with(0, 1);
    if (y == 0) m &= ~slots_with(1, -1);
    if (y + 1 == F.ny) m &= ~slots_with(1, 1);
    if (z == 0) m &= ~slots_with(2, -1);
    if (z + 1 == F.nz) m &= ~slots_with(2, 1);
    return m;
}

// Slots whose paths the event lists follow: the lower link of a join saddle
// (descent to minima) and the upper link of a split saddle (ascent to maxima).
__device__ __forceinline__ void event_sides(const Dev &D, uint32_t d, uint32_t valid, uint32_t &Ls, uint32_t &Us)
{
    const uint32_t L = (d >> D_MASK_SHIFT) & 0x3FFFu, U = valid & ~L;
    Ls = multi_bit(D.multi, L) ? L : 0u;
    Us = multi_bit(D.multi, U) ? U : 0u;
}

// Distinct path ends through the slots in `side` (E: the links of that
// direction), appended to ext[n0 ...]; the f-selection (largest minimum with
// up = 0, smallest maximum with up = 1, ties by index) is moved to ext[n0].
// Returns their number, 0 when fewer than two.
__device__ __forceinline__ uint32_t path_ends(const FieldDesc &F, const uint32_t *E, uint64_t a, uint32_t side,
                                              const long long *off, int up, uint32_t *ext, uint32_t n0)
{
    uint32_t c = 0, bi = 0, b = 0;
    float bf = 0.0f;
    for (uint32_t m = side; m; m &= m - 1) {
        const uint32_t e = (E[a + off[__ffs(m) - 1]] & ~EV_DONE) - (uint32_t)F.vbase;
        bool dup = false;
        for (uint32_t i = 0; i < c; i++) dup |= ext[n0 + i] == e;
        if (dup) continue;
        const float fe = F.f[e];
        const bool better = c == 0 || (up ? (fe < bf || (fe == bf && e < b)) : (bf < fe || (bf == fe && b < e)));
        if (better) {
            bi = c;
            bf = fe;
            b = e;
        }
        ext[n0 + c++] = e;
    }
    if (c < 2) return 0;
    ext[n0 + bi] = ext[n0];
    ext[n0] = b;
    return c;
}

// The listed saddles in grid order: a warp takes 32 consecutive words of the
// listed-point bitmap (chunk ch; a chunk never straddles two fields), numbers
// their set bits and hands them to its lanes 32 at a time; body(F, fid, x, y,
// z, t, have) runs for each (every lane calls it the same number of times;
// `have` is false for an idle lane).  The field's neighbour offsets are in
// off (per warp, shared memory).
template <class Body>
__device__ __forceinline__ void for_listed_saddles(const Dev &D, long long *off, Body body)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long nchunks = (D.total_w + 31) / 32;
    const unsigned long long w0 = ((unsigned long long)blockIdx.x * CTA + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * CTA) >> 5;
    for (unsigned long long ch = w0; ch < nchunks; ch += nw) {
        const uint64_t w = ch * 32 + lane;
        const uint32_t word = w < D.total_w ? D.cpwords[w] : 0u;
        if (!__any_sync(0xffffffffu, word != 0)) {
            body(ch, (const FieldDesc *)nullptr, 0u, 0u, 0u, 0u, 0u, 0u, false);
            continue;
        }
        const uint32_t fid = field_of_word(D, ch * 32, 0, D.nfields);
        const FieldDesc &F = D.fields[fid];
        if (lane < 14) off[lane] = rank_offset(F, rank_of(lane));
        __syncwarp();
        const uint32_t cw = __popc(word);
        uint32_t incl = cw;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t excl = incl - cw;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t k = base + lane;
            int src = 0;  // the last lane whose first number is <= k
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint32_t pe = __shfl_sync(0xffffffffu, excl, src + step);
                if (pe <= k) src += step;
            }
            const uint32_t rword = __shfl_sync(0xffffffffu, word, src);
            const uint32_t rpre = __shfl_sync(0xffffffffu, excl, src);
            const bool have = k < total;
            uint32_t x = 0, y = 0, z = 0, t = 0;
            if (have) {
                const uint32_t wl = (uint32_t)(ch * 32 + src - F.wbase);
                const uint32_t row = fdiv(wl, F.div_tnx), wx = wl - row * F.tnx;
                z = fdiv(row, F.div_ny);
                y = row - z * F.ny;
                x = wx * TX + (uint32_t)nth_set_bit(rword, (int)(k - rpre));
                t = (uint32_t)(((uint64_t)z * F.ny + y) * F.nx + x);
            }
            body(ch, &F, fid, x, y, z, t, base, have);
        }
        __syncwarp();
    }
}

// Exclusive warp prefix of v; *sum = the warp total.
__device__ __forceinline__ uint32_t warp_excl(uint32_t v, uint32_t *sum)
{
    const int lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *sum = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// WRITE = 0: per chunk, the room its saddles' lists may need (the number of
// slots the lists follow), into room[ch].  WRITE = 1: with room_off the
// exclusive prefix sums of those numbers, each saddle's list goes to its room
// (ev_start, ev_cnt at its position q in the sorted order), cp_rank[e] (zero
// for every extremum after the set-up check) counts the saddles linked to
// extremum e, and ls->ev_cursor[1] the list entries written.
template <int WRITE>
__global__ void __launch_bounds__(CTA) k_ev_lists(Dev D, const uint32_t *E, uint32_t *room,
                                                  const unsigned long long *room_off, uint32_t *list, uint32_t *start,
                                                  uint16_t *cnt)
{
    __shared__ long long s_off[WARPS][14];
    const int lane = threadIdx.x & 31;
    long long *off = s_off[threadIdx.x >> 5];
    uint32_t run = 0, written = 0;
    unsigned long long cur = ~0ull;
    for_listed_saddles(D, off, [&](unsigned long long ch, const FieldDesc *F, uint32_t fid, uint32_t x, uint32_t y,
                                   uint32_t z, uint32_t t, uint32_t base, bool have) {
        if (ch != cur) {  // a new chunk (warp-uniform)
            if (!WRITE && cur != ~0ull && lane == 0) room[cur] = run;
            cur = ch;
            run = 0;
        }
        if (!F) return;
        uint32_t d = 0, Ls = 0, Us = 0;
        if (have) {
            d = D.desc[F->vbase + t];
            event_sides(D, d, valid_slots(*F, x, y, z), Ls, Us);
        }
        const uint32_t need = __popc(Ls) + __popc(Us);
        uint32_t tot;
        const uint32_t ex = warp_excl(need, &tot);
        if (WRITE && have) {
            const uint64_t a = F->vbase + t;
            uint32_t ext[14];
            const uint32_t c0 = Ls ? path_ends(*F, E, a, Ls, off, 0, ext, 0) : 0u;
            const uint32_t c1 = Us ? path_ends(*F, E + D.total_v, a, Us, off, 1, ext, c0) : 0u;
            const unsigned long long q = D.fst[fid].cp_base + D.cp_rank[a];
            const unsigned long long pos = room_off[ch] + run + ex;
            for (uint32_t i = 0; i < c0 + c1; i++) {
                list[pos + i] = ext[i];
                atomicAdd(&D.cp_rank[F->vbase + ext[i]], 1u);
            }
            start[q] = (uint32_t)pos;
            cnt[q] = (uint16_t)(c0 | (c1 << 8));
            written += c0 + c1;
        }
        run += tot;
    });
    if (!WRITE && cur != ~0ull && lane == 0) room[cur] = run;
    if (WRITE) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, written);
        if (lane == 0 && v) atomicAdd(&D.ls->ev_cursor[1], (unsigned long long)v);
    }
}

// Every extremum with linked saddles gets its run in ev_radj: the count
// first (a fill cursor until k_ev_fill), then the saddles; cp_rank[e] = the
// run's position, from 1 on (0 stays "no linked saddle").
__global__ void __launch_bounds__(CTA) k_ev_alloc(Dev D, uint32_t *radj)
{
    __shared__ uint32_t sw[WARPS];
    __shared__ unsigned long long sbase;
    for_tile_vertices(D, [&](uint32_t, const FieldDesc &F, uint32_t t, uint32_t, uint32_t, uint32_t, bool in) {
        uint32_t deg = 0;
        const uint64_t a = F.vbase + t;
        if (in) {
            const uint32_t d = D.desc[a];
            if (!(d & D_CP) && ((d & 15u) == 7u || ((d >> D_DN_SHIFT) & 15u) == 7u)) deg = D.cp_rank[a];
        }
        const unsigned long long h = 1 + block_reserve(deg ? deg + 1 : 0u, &D.ls->ev_cursor[2], sw, &sbase);
        if (deg) {
            radj[h] = 0;
            D.cp_rank[a] = (uint32_t)h;
        }
    });
}

// The saddles of each extremum, in grid order of the saddles.
__global__ void __launch_bounds__(CTA) k_ev_fill(Dev D, uint32_t *radj)
{
    __shared__ long long s_off[WARPS][14];
    long long *off = s_off[threadIdx.x >> 5];
    for_listed_saddles(D, off, [&](unsigned long long, const FieldDesc *F, uint32_t fid, uint32_t, uint32_t,
                                   uint32_t, uint32_t t, uint32_t, bool have) {
        if (!have) return;
        const uint64_t a = F->vbase + t;
        const unsigned long long q = D.fst[fid].cp_base + D.cp_rank[a];
        const uint32_t c = D.ev_cnt[q];
        if (!c) return;
        const uint32_t *l = D.ev_list + D.ev_start[q];
        const uint32_t n = (c & 255u) + (c >> 8);
        for (uint32_t i = 0; i < n; i++) {
            const uint32_t h = D.cp_rank[F->vbase + l[i]];
            const uint32_t slot = atomicAdd(&radj[h], 1u);
            radj[h + 1 + slot] = (uint32_t)q;
        }
    });
}

// ------------------------------------------------------------ bookkeeping
// Per-field end of a pass by one block of NT threads: a field with requests
// this pass counts an iteration, the others are done; sets the loop flag and
// the graph conditional.  The field state is read through volatile accesses:
// in the fused pass kernel other blocks wrote it earlier in the same launch.
template <int NT>
__device__ __forceinline__ void book_fields(const Dev &D, cudaGraphConditionalHandle h, int use_graph)
{
    __shared__ uint32_t s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    // a bounded wait ran out: stop every field (the call reports it)
    const bool fault = *reinterpret_cast<volatile uint32_t *>(&D.ls->fault) != 0;
    for (uint32_t f = threadIdx.x; f < D.nfields; f += NT) {
        volatile FieldState *S = &D.fst[f];
        if (S->done) continue;
        if (S->err || S->capped || fault) {
            S->done = 1;
            continue;
        }
        if (S->had_req) {
            S->iterations += 1;
            S->had_req = 0;
            s_any = 1;
        } else {
            S->done = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        LoopState *L = D.ls;
        L->pass += 1;
        L->any_active = s_any;
        if (use_graph) cudaGraphSetConditional(h, s_any ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(CTA) k_book(Dev D, cudaGraphConditionalHandle h, int use_graph)
{
    book_fields<CTA>(D, h, use_graph);
}

// Sets the loop flag (and graph conditional) from the per-field state.
__global__ void __launch_bounds__(SMALL_NT) k_loop_flag(Dev D, cudaGraphConditionalHandle h, int use_graph)
{
    __shared__ uint32_t s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (uint32_t f = threadIdx.x; f < D.nfields; f += blockDim.x)
        if (!D.fst[f].done) s_any = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        D.ls->any_active = s_any;
        if (use_graph) cudaGraphSetConditional(h, s_any ? 1u : 0u);
    }
}

// ------------------------------------------------------------ fused pass
// Barrier across all blocks of the fused pass kernel, which is launched
// cooperatively (every block resident).  The wait is bounded: when it runs
// out, the block sets the fault flag, stops the graph loop and gets false
// (the caller returns; blocks still waiting run out the same way).
__device__ __forceinline__ bool grid_barrier(const Dev &D, cudaGraphConditionalHandle h)
{
    __shared__ uint32_t s_ok;
    __threadfence();  // this block's writes before the arrival
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *gen = &D.ls->bar_gen;
        const uint32_t g0 = *gen;
        __threadfence();  // the generation is read before the arrival
        uint32_t ok = 1;
        if (atomicAdd(&D.ls->bar_count, 1u) == gridDim.x - 1) {
            D.ls->bar_count = 0;  // everyone has arrived; nobody arrives again before the generation moves
            __threadfence();
            atomicAdd(&D.ls->bar_gen, 1u);
        } else {
            for (uint32_t i = 0; *gen == g0; i++) {
                if (i == (1u << 24)) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!ok) {
            atomicOr(&D.ls->fault, 1u);
            cudaGraphSetConditional(h, 0u);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One frontier pass in one launch, the body of the fused graph loop
// (EXACTZ_MODE_FUSED): the vertex check (rules R1, R2) and the CP-pair check
// (R3) of every block, a grid barrier, the bounded edit, and the bookkeeping
// by the last block to finish its edits.  The same phases and results as the
// graph loop's four kernels.
__global__ void __launch_bounds__(SCTA, 6) k_pass(Dev D, cudaGraphConditionalHandle h)
{
    stencil_tiles<SM_CHECK_LIST>(D, nullptr, nullptr, 0, 0, nullptr, 0);
    pairs_body<PM_LIST, SCTA>(D, 0, nullptr, nullptr, 0);
    if (!grid_barrier(D, h)) return;
    apply_tiles<AM_FRONTIER, SCTA / 32>(D);
    __shared__ uint32_t s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&D.ls->pass_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();  // every block's edits and counters before the bookkeeping reads them
    if (threadIdx.x == 0) D.ls->pass_done = 0;
    book_fields<SCTA>(D, h, 1);
}

// ------------------------------------------------------------ status
__global__ void __launch_bounds__(SMALL_NT) k_status(Dev D, FieldSet FS)
{
    for (uint32_t j = threadIdx.x + blockIdx.x * blockDim.x; j < FS.n; j += blockDim.x * gridDim.x) {
        FieldState *S = &D.fst[FS.fids[j]];
        if (S->err & ERR_NONFINITE) S->status = (uint32_t)-2;
        else if (S->err & ERR_BOUND) S->status = (uint32_t)-3;
        else if (S->capped) S->status = ST_ITER_LIMIT;
        else S->status = (S->pinned_res ? ST_STUCK : ST_CONVERGED);
    }
}

// ------------------------------------------------------------ edit list
constexpr int EPT = VBLOCK / CTA;  // arena vertices per thread

__device__ __forceinline__ uint32_t field_of_vertex(const Dev &D, uint64_t v, uint32_t lo, uint32_t hi)
{
    hi -= 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (D.fields[mid].vbase <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(CTA) k_edit_count(Dev D, FieldSet FS)
{
    const uint64_t vblk0 = FS.vblk0;
    __shared__ uint32_t sw[WARPS];
    __shared__ uint32_t s_lossless;
    if (threadIdx.x == 0) s_lossless = 0;
    const uint64_t v0 = (vblk0 + blockIdx.x) * VBLOCK;
    const uint32_t fid = field_of_vertex(D, v0, FS.fid0, FS.fid1);
    const uint32_t N = D.fields[fid].N;
    const uint64_t b = v0 + threadIdx.x * EPT;
    uint32_t c = 0, l = 0;
    const uint4 *dp = reinterpret_cast<const uint4 *>(D.desc + b);
#pragma unroll
    for (int j = 0; j < EPT / 4; j++) {
        const uint4 w = dp[j];
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t kk = ws[u] >> D_K_SHIFT;
            c += kk != 0;
            l += kk == N + 1;
        }
    }
    __syncthreads();
    if (l) atomicAdd(&s_lossless, l);
    uint32_t ex;
    const uint32_t tot = block_excl_scan_n<CTA>(c, ex, sw);
    if (threadIdx.x == 0) {
        D.blk[blockIdx.x] = tot;
        if (tot) atomicAdd(&D.fst[fid].n_edits, (unsigned long long)tot);
        if (s_lossless) atomicAdd(&D.fst[fid].n_lossless, (unsigned long long)s_lossless);
    }
}

__global__ void __launch_bounds__(CTA) k_edit_write(Dev D, FieldSet FS)
{
    const uint64_t vblk0 = FS.vblk0;
    __shared__ uint32_t sw[WARPS];
    const uint64_t v0 = (vblk0 + blockIdx.x) * VBLOCK;
    const uint32_t fid = field_of_vertex(D, v0, FS.fid0, FS.fid1);
    const FieldDesc &F = D.fields[fid];
    if (!F.edits) return;
    const uint32_t N = F.N;
    const uint64_t b = v0 + threadIdx.x * EPT;
    uint32_t kks[EPT];
    uint32_t c = 0;
    const uint4 *dp = reinterpret_cast<const uint4 *>(D.desc + b);
#pragma unroll
    for (int j = 0; j < EPT / 4; j++) {
        const uint4 w = dp[j];
        kks[4 * j + 0] = w.x >> D_K_SHIFT;
        kks[4 * j + 1] = w.y >> D_K_SHIFT;
        kks[4 * j + 2] = w.z >> D_K_SHIFT;
        kks[4 * j + 3] = w.w >> D_K_SHIFT;
    }
#pragma unroll
    for (int j = 0; j < EPT; j++) c += kks[j] != 0;
    uint32_t ex;
    block_excl_scan_n<CTA>(c, ex, sw);
    const unsigned long long fbase = D.blk_off[F.vbase / VBLOCK - vblk0];
    unsigned long long pos = D.blk_off[blockIdx.x] + ex - fbase;
    if (!c) return;
    // a reflected field (increasing edits): its records in the caller's
    // coordinates and order
    const unsigned long long ne = F.mirror ? D.fst[fid].n_edits : 0ull;
#pragma unroll
    for (int j = 0; j < EPT; j++) {
        const uint32_t kk = kks[j];
        if (!kk) continue;
        const unsigned long long at = F.mirror ? ne - 1 - pos : pos;
        if (at < F.edits_cap) {
            const uint64_t t = b + j - F.vbase;
            EditRec r;
            r.idx = F.mirror ? F.n - 1 - t : t;
            r.value = F.mirror ? unreflect(F.g[t], kk) : F.g[t];
            r.k = (uint8_t)kk;
            r.lossless = kk == N + 1;
            r.reserved = 0;
            F.edits[at] = r;
        }
        pos++;
    }
}

// Increasing edits by reflection: dst[v] = -src[n-1-v].
__global__ void __launch_bounds__(CTA) k_reflect_in(const float *src, float *dst, uint64_t n)
{
    for (uint64_t v = (uint64_t)blockIdx.x * CTA + threadIdx.x; v < n; v += (uint64_t)gridDim.x * CTA)
        dst[v] = -src[n - 1 - v];
}

// The result back in the caller's coordinates, in place: g[v] <-> -g[n-1-v];
// an edited value never becomes -0 (see unreflect).
__global__ void __launch_bounds__(CTA) k_reflect_out(float *g, const uint32_t *desc, uint64_t n)
{
    const uint64_t half = (n + 1) / 2;
    for (uint64_t i = (uint64_t)blockIdx.x * CTA + threadIdx.x; i < half; i += (uint64_t)gridDim.x * CTA) {
        const uint64_t j = n - 1 - i;
        const float a = g[i], b = g[j];
        const uint32_t ki = desc[j] >> D_K_SHIFT, kj = desc[i] >> D_K_SHIFT;  // k of caller vertices i and j
        g[i] = unreflect(b, ki);
        if (j != i) g[j] = unreflect(a, kj);
    }
}

// g of the fields kept in a padded copy during the passes, back in the
// field's own layout: one tile per warp, lane x of each of the tile's rows.
__global__ void __launch_bounds__(CTA) k_unmirror(Dev D)
{
    const int lane = threadIdx.x & 31;
    for (uint64_t tile = (uint64_t)blockIdx.x * WARPS + (threadIdx.x >> 5); tile < D.total_tiles;
         tile += (uint64_t)gridDim.x * WARPS) {
        const uint32_t fid = field_of_tile(D, (uint32_t)tile);
        const FieldDesc &F = D.fields[fid];
        const float *gm = F.gm;
        if (!gm) continue;
        const TileGeo G = tile_geo_of(D, (uint32_t)tile, fid);
        const uint32_t x = (uint32_t)G.x0 + lane, nx = F.nx, ny = F.ny, nz = F.nz, pitch = F.pitch;
        if (x >= nx) continue;
        float *g = F.g;
        float v[ROWS];  // all of the tile's rows in flight before the first store
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            const uint32_t y = (uint32_t)G.y0 + r % TY, z = (uint32_t)G.z0 + r / TY;
            v[r] = (y < ny && z < nz) ? gm[((uint64_t)z * ny + y) * pitch + x] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            const uint32_t y = (uint32_t)G.y0 + r % TY, z = (uint32_t)G.z0 + r / TY;
            if (y < ny && z < nz) g[((uint64_t)z * ny + y) * nx + x] = v[r];
        }
    }
}

// ------------------------------------------------------------ edit stream (Sec. 3.3; storage accounting)
// The stored form of a result: one edit-count byte per vertex (0..N steps of
// Delta, N+1 = the lossless bound) and the lossless values in index order.
// Blocks take SB consecutive items, SPT per thread.
constexpr int SPT = 16;
constexpr int SB = CTA * SPT;

// kcodes[idx] = k for every edit (kcodes cleared beforehand).  An edit list
// that is not strictly ascending, names a vertex outside [0, n), or has a k
// outside 1..N+1 or a lossless flag that disagrees with k = N+1 sets *bad and
// writes nothing for that record.
__global__ void __launch_bounds__(CTA) k_stream_kcodes(const EditRec *edits, uint64_t ne, uint64_t n, uint32_t N,
                                                       uint8_t *kcodes, int *bad)
{
    for (uint64_t i = (uint64_t)blockIdx.x * CTA + threadIdx.x; i < ne; i += (uint64_t)gridDim.x * CTA) {
        const EditRec r = edits[i];
        const bool ok = r.idx < n && r.k >= 1 && r.k <= N + 1 && (r.lossless != 0) == (r.k == N + 1) &&
                        (i + 1 == ne || edits[i + 1].idx > r.idx);
        if (ok) kcodes[r.idx] = r.k;
        else *bad = 1;
    }
}

// Lossless items per block: edits with the lossless flag (from_codes = 0), or
// vertices whose code is N + 1 (from_codes = 1, also flags codes above N + 1).
__global__ void __launch_bounds__(CTA) k_stream_count(const EditRec *edits, const uint8_t *kcodes, uint64_t n,
                                                      uint32_t N, int from_codes, uint32_t *blk, int *bad)
{
    __shared__ uint32_t sw[WARPS];
    const uint64_t b = (uint64_t)blockIdx.x * SB + (uint64_t)threadIdx.x * SPT;
    uint32_t c = 0;
    bool wrong = false;
    for (int j = 0; j < SPT; j++) {
        const uint64_t i = b + j;
        if (i >= n) break;
        if (from_codes) {
            const uint32_t k = kcodes[i];
            c += k == N + 1;
            wrong |= k > N + 1;
        } else {
            c += edits[i].lossless != 0;
        }
    }
    if (wrong) *bad = 1;
    uint32_t ex;
    const uint32_t tot = block_excl_scan_n<CTA>(c, ex, sw);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

// Encode: the lossless values of the edit list, in its (index) order.
__global__ void __launch_bounds__(CTA) k_stream_lossless(const EditRec *edits, uint64_t ne,
                                                         const unsigned long long *blk_off, float *lossless)
{
    __shared__ uint32_t sw[WARPS];
    const uint64_t b = (uint64_t)blockIdx.x * SB + (uint64_t)threadIdx.x * SPT;
    uint32_t c = 0;
    for (int j = 0; j < SPT && b + j < ne; j++) c += edits[b + j].lossless != 0;
    uint32_t ex;
    block_excl_scan_n<CTA>(c, ex, sw);
    unsigned long long pos = blk_off[blockIdx.x] + ex;
    for (int j = 0; j < SPT && b + j < ne; j++)
        if (edits[b + j].lossless) lossless[pos++] = edits[b + j].value;
}

// Decode: g_i = f_hat_i after k_i steps of fl(g - Delta) (fl(g + Delta) with
// inc), or the next lossless value.
__global__ void __launch_bounds__(CTA) k_stream_decode(const float *fhat, const uint8_t *kcodes, const float *lossless,
                                                       uint64_t n, uint32_t N, float delta, int inc,
                                                       const unsigned long long *blk_off, float *g)
{
    __shared__ uint32_t sw[WARPS];
    const uint64_t b = (uint64_t)blockIdx.x * SB + (uint64_t)threadIdx.x * SPT;
    uint32_t c = 0;
    for (int j = 0; j < SPT && b + j < n; j++) c += kcodes[b + j] == N + 1;
    uint32_t ex;
    block_excl_scan_n<CTA>(c, ex, sw);
    unsigned long long pos = blk_off[blockIdx.x] + ex;
    for (int j = 0; j < SPT && b + j < n; j++) {
        const uint64_t i = b + j;
        const uint32_t k = kcodes[i];
        float v = fhat[i];
        if (k == N + 1) {
            v = lossless[pos++];
        } else if (k <= N) {
            for (uint32_t s = 0; s < k; s++) v = inc ? __fadd_rn(v, delta) : __fsub_rn(v, delta);
        }
        g[i] = v;
    }
}

// ------------------------------------------------------------ launch wrappers
static int sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

static unsigned grid_for(uint64_t items, int per_block, int cap_mult)
{
    uint64_t g = (items + per_block - 1) / per_block;
    uint64_t cap = (uint64_t)sms() * cap_mult;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

__global__ void __launch_bounds__(SMALL_NT) k_fill_u32(uint32_t *p, uint32_t v, uint64_t n)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

void launch_fill_u32(uint32_t *p, uint32_t v, uint64_t n, cudaStream_t s)
{
    if (n) k_fill_u32<<<grid_for(n, SMALL_NT, 4), SMALL_NT, 0, s>>>(p, v, n);
}

int device_sms() { return sms(); }

void launch_setup(const Dev &D, const SetupRange &R, cudaStream_t s)
{
    k_stencil<SM_SETUP><<<grid_for(R.tile1 - R.tile0, 1, 8), SCTA, 0, s>>>(D, nullptr, nullptr, R.tile0, R.tile1,
                                                                          nullptr, 0);
}
void launch_check_all(const Dev &D, cudaStream_t s)
{
    k_stencil<SM_CHECK_ALL><<<grid_for(D.total_tiles, 1, D.tun.stencil_bps), SCTA, 0, s>>>(
        D, nullptr, nullptr, 0, D.total_tiles, nullptr, 0);
}
void launch_check_list(const Dev &D, cudaStream_t s)
{
    k_stencil<SM_CHECK_LIST><<<grid_for(D.total_tiles, 1, D.tun.stencil_bps), SCTA, 0, s>>>(
        D, nullptr, nullptr, 0, 0, nullptr, 0);
}
void launch_check_pinned(const Dev &D, const FieldSet &FS, cudaStream_t s)
{
    k_stencil<SM_PINNED><<<grid_for(D.total_tiles, 1, 16), SCTA, 0, s>>>(D, nullptr, nullptr, 0, 0, FS.fids, FS.n);
}
void launch_classify(const Dev &D, uint32_t *desc_out, uint8_t *type_out, cudaStream_t s)
{
    k_stencil<SM_CLASSIFY><<<grid_for(D.total_tiles, 1, 16), SCTA, 0, s>>>(D, desc_out, type_out, 0, D.total_tiles,
                                                                         nullptr, 0);
}

void launch_cp_compact(const Dev &D, const SetupRange &R, cudaStream_t s)
{
    const unsigned nb = (unsigned)R.nwblk;
    k_cp_count<<<nb, CTA, 0, s>>>(D, R.wblk0);
    k_scan_u32<<<1, SCAN_NT, 0, s>>>(D.blk, D.blk_off, R.nwblk, R.cp_count);
    k_cp_write<<<nb, CTA, 0, s>>>(D, R);
    k_cp_ncp<<<(R.fid1 - R.fid0 + SMALL_NT - 1) / SMALL_NT, SMALL_NT, 0, s>>>(D, R);
}

// LSD passes of one sort: four 8-bit digits of the value key, then the digits
// of the field id when the range holds more than one field.
int sort_passes(uint32_t fid0, uint32_t fid1)
{
    int p = 4;
    if (fid1 - fid0 > 1) {
        const uint32_t top = fid1 - 1;
        p += 1;
        if (top > 255) p += 1;
        if (top > 65535) p += 1;
    }
    return p;
}

void launch_cp_sort(const Dev &D, const SetupRange &R, cudaStream_t s)
{
    const int P = sort_passes(R.fid0, R.fid1);
    const unsigned B = D.sort_blocks;
    int src = 0;
    for (int p = 0; p < P; p++) {
        const int dst = src ^ 1;
        k_sort_hist<<<B, RADIX, 0, s>>>(D, p, D.cp_key[src] + R.cp0, D.cp_ent[src] + R.cp0, R.cp_count);
        k_scan_inplace_u32<<<1, SCAN_NT, 0, s>>>(D.hist, (uint64_t)RADIX * B);
        k_sort_scatter<<<B, RADIX, 0, s>>>(D, p, D.cp_key[src] + R.cp0, D.cp_ent[src] + R.cp0,
                                           D.cp_key[dst] + R.cp0, D.cp_ent[dst] + R.cp0, p == P - 1, R.cp_count,
                                           R.cp0);
        src = dst;
    }
}

void launch_pairs_all(const Dev &D, const SetupRange &R, cudaStream_t s)
{
    k_pairs<PM_ALL><<<sms() * 8, CTA, 0, s>>>(D, R.cp0, R.cp_count, nullptr, 0);
}
void launch_pairs_list(const Dev &D, cudaStream_t s)
{
    k_pairs<PM_LIST><<<sms() * D.tun.pairs_bps, CTA, 0, s>>>(D, 0, nullptr, nullptr, 0);
}
void launch_pairs_pinned(const Dev &D, const FieldSet &FS, cudaStream_t s)
{
    k_pairs<PM_PINNED><<<sms() * 4, CTA, 0, s>>>(D, 0, nullptr, FS.fids, FS.n);
}

void launch_ev_init(const Dev &D, uint32_t *E, cudaStream_t s)
{
    k_ev_init<<<grid_for(D.total_tiles, 1, 8), CTA, 0, s>>>(D, E);
}
void launch_ev_jump(const Dev &D, uint32_t *E, uint8_t *tdone, cudaStream_t s)
{
    k_ev_jump<<<grid_for(D.total_tiles, 1, 8), CTA, 0, s>>>(D, E, tdone);
}
void launch_ev_lists(const Dev &D, const uint32_t *E, int write, uint32_t *room,
                     const unsigned long long *room_off, uint32_t *list, uint32_t *start, uint16_t *cnt,
                     cudaStream_t s)
{
    if (write) k_ev_lists<1><<<sms() * 8, CTA, 0, s>>>(D, E, room, room_off, list, start, cnt);
    else k_ev_lists<0><<<sms() * 8, CTA, 0, s>>>(D, E, room, room_off, list, start, cnt);
}
void launch_scan_u32(const uint32_t *in, unsigned long long *out, uint64_t n, unsigned long long *total,
                     cudaStream_t s)
{
    k_scan_u32<<<1, SCAN_NT, 0, s>>>(in, out, n, total);
}
void launch_ev_reverse(const Dev &D, uint32_t *radj, cudaStream_t s)
{
    k_ev_alloc<<<grid_for(D.total_tiles, 1, 8), CTA, 0, s>>>(D, radj);
    k_ev_fill<<<sms() * 8, CTA, 0, s>>>(D, radj);
}

void launch_apply(const Dev &D, int frontier, cudaStream_t s)
{
    if (frontier) k_apply_tiles<AM_FRONTIER><<<grid_for(D.total_tiles, WARPS, D.tun.apply_bps), CTA, 0, s>>>(D);
    else k_apply_tiles<AM_PLAIN><<<grid_for(D.total_tiles, WARPS, D.tun.apply_bps), CTA, 0, s>>>(D);
}
void launch_book(const Dev &D, cudaGraphConditionalHandle h, int use_graph, cudaStream_t s)
{
    k_book<<<1, CTA, 0, s>>>(D, h, use_graph);
}
cudaError_t pass_grid(unsigned *grid)
{
    int nb = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pass, SCTA, 0);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorCooperativeLaunchTooLarge;
    *grid = (unsigned)(nb * sms());  // every block resident
    return cudaSuccess;
}
cudaError_t launch_pass(const Dev &D, cudaGraphConditionalHandle h, unsigned grid, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(SCTA);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pass, D, h);
}
void launch_loop_flag(const Dev &D, cudaGraphConditionalHandle h, int use_graph, cudaStream_t s)
{
    k_loop_flag<<<1, SMALL_NT, 0, s>>>(D, h, use_graph);
}
void launch_finish(const Dev &D, const FieldSet &FS, cudaStream_t s)
{
    k_apply_tiles<AM_COUNT><<<grid_for(D.total_tiles, WARPS, 16), CTA, 0, s>>>(D);
    k_status<<<(FS.n + SMALL_NT - 1) / SMALL_NT, SMALL_NT, 0, s>>>(D, FS);
}
void launch_edit_list(const Dev &D, const FieldSet &FS, int write, cudaStream_t s)
{
    const unsigned nb = (unsigned)FS.nvblk;
    k_edit_count<<<nb, CTA, 0, s>>>(D, FS);
    if (write) {
        k_scan_u32<<<1, SCAN_NT, 0, s>>>(D.blk, D.blk_off, FS.nvblk, nullptr);
        k_edit_write<<<nb, CTA, 0, s>>>(D, FS);
    }
}

unsigned stream_blocks(uint64_t items) { return (unsigned)((items + SB - 1) / SB); }
void launch_stream_kcodes(const EditRec *edits, uint64_t ne, uint64_t n, uint32_t N, uint8_t *kcodes, int *bad,
                          cudaStream_t s)
{
    if (ne) k_stream_kcodes<<<grid_for(ne, CTA, 8), CTA, 0, s>>>(edits, ne, n, N, kcodes, bad);
}
void launch_stream_count(const EditRec *edits, const uint8_t *kcodes, uint64_t n, uint32_t N, int from_codes,
                         uint32_t *blk, int *bad, cudaStream_t s)
{
    if (n) k_stream_count<<<stream_blocks(n), CTA, 0, s>>>(edits, kcodes, n, N, from_codes, blk, bad);
}
void launch_stream_lossless(const EditRec *edits, uint64_t ne, const unsigned long long *blk_off, float *lossless,
                            cudaStream_t s)
{
    if (ne) k_stream_lossless<<<stream_blocks(ne), CTA, 0, s>>>(edits, ne, blk_off, lossless);
}
void launch_stream_decode(const float *fhat, const uint8_t *kcodes, const float *lossless, uint64_t n, uint32_t N,
                          float delta, int inc, const unsigned long long *blk_off, float *g, cudaStream_t s)
{
    if (n) k_stream_decode<<<stream_blocks(n), CTA, 0, s>>>(fhat, kcodes, lossless, n, N, delta, inc, blk_off, g);
}

void launch_reflect_in(const float *src, float *dst, uint64_t n, cudaStream_t s)
{
    k_reflect_in<<<grid_for(n, CTA, 8), CTA, 0, s>>>(src, dst, n);
}
void launch_unmirror(const Dev &D, cudaStream_t s)
{
    k_unmirror<<<grid_for(D.total_tiles, WARPS, 8), CTA, 0, s>>>(D);
}
void launch_reflect_out(float *g, const uint32_t *desc, uint64_t n, cudaStream_t s)
{
    k_reflect_out<<<grid_for((n + 1) / 2, CTA, 8), CTA, 0, s>>>(g, desc, n);
}

}  // namespace exz
