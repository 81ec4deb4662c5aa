// exz_kernels.cu -- sm_103a kernels of the EXaCTz correction (Algorithm 1).
//
//   k_stencil<SETUP>   per-vertex descriptor of f (steepest up/down rank, lower
//                      link mask, saddle / critical flags; Sec. 3.2, Sec. 4.2),
//                      input validation, g := f_hat, k := 0, critical-point
//                      bitmap, and the first pass's EG / saddle-link checks.
//   k_stencil<CHECK_*> EG constraints and saddle-link rule on the edited field
//                      g (Sec. 4.2) for all tiles or the tiles touched by the
//                      previous pass; emits decrease requests.
//   k_cp_*             ordered compaction of critical points; stable LSD radix
//                      sort by (field, value key) -> f's global CP order (Sec. 4.3).
//   k_pairs            reformulated event constraint: adjacent CP pairs whose
//                      g-order is reversed (Sec. 4.3).
//   k_apply            bounded monotone edit (Sec. 3.3) of each requested vertex
//                      once, frontier marking for the next pass.
//   k_book             per-field convergence bookkeeping, device-side loop flag.
//   k_finish/k_status  residual violations and final status.
//   k_edit_*           ordered compaction of the edit list.
//
// Requests are deduplicated by an atomic bitmap over the arena; a vertex is
// edited at most once per pass (synchronous semantics, Sec. 4.4 proof).
#include <cmath>
#include <cstdio>

#include "exz_common.cuh"
#include "exz_launch.h"

namespace exz {

enum { SM_SETUP = 0, SM_CHECK_ALL = 1, SM_CHECK_LIST = 2, SM_PINNED = 3, SM_CLASSIFY = 4 };
enum { EM_FIRST = 0, EM_NORMAL = 1, EM_PINNED = 2 };

constexpr int QCAP = 1024;

__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// ------------------------------------------------------------ emission
struct EmitQ {
    unsigned long long e[QCAP];
    uint32_t n;
    unsigned long long base;
};

__device__ __forceinline__ void q_push(EmitQ &q, const Dev &D, unsigned long long e)
{
    uint32_t p = atomicAdd(&q.n, 1u);
    if (p < QCAP) {
        q.e[p] = e;
    } else {
        unsigned long long gp = atomicAdd(&D.ls->req_count, 1ull);
        D.req_list[gp] = e;
    }
}

// All threads of the block must call this.
__device__ __forceinline__ void q_flush(EmitQ &q, const Dev &D)
{
    __syncthreads();
    uint32_t n = min(q.n, (uint32_t)QCAP);
    if (threadIdx.x == 0 && n) q.base = atomicAdd(&D.ls->req_count, (unsigned long long)n);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n; j += CTA) D.req_list[q.base + j] = q.e[j];
    __syncthreads();
    if (threadIdx.x == 0) q.n = 0;
}

// Request a decrease of local vertex t of field fid (deduplicated).
template <int EM>
__device__ __forceinline__ void emit(const Dev &D, EmitQ &q, uint32_t fid, uint64_t vbase, uint32_t N,
                                     uint64_t t)
{
    uint64_t gid = vbase + t;
    if (EM == EM_NORMAL) {
        if (D.k[gid] > N) return;  // pinned at the lossless bound
    } else if (EM == EM_PINNED) {
        if (D.k[gid] <= N) return;
    }
    uint32_t bit = 1u << (gid & 31);
    uint32_t *w = &D.reqbits[gid >> 5];
    if (__ldcg(w) & bit) return;
    uint32_t old = atomicOr(w, bit);
    if (old & bit) return;
    q_push(q, D, ((unsigned long long)fid << LOCAL_BITS) | t);
}

// ------------------------------------------------------------ stencil core
// Steepest-ascent / -descent rank and lower-link mask of the vertex at smem
// index c.  Out-of-domain cells hold NaN: never selected, never "lower".
struct Stn {
    uint32_t up, dn, mask, valid;
};

template <bool INTERIOR>
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
    uint32_t valid = 0x3FFFu;
    if (!INTERIOR) {
        valid = 0;
#pragma unroll
        for (int r = 0; r < 15; r++)
            if (r != 7) valid |= (v[r] == v[r]) ? (1u << slot_of(r)) : 0u;
    }
    return Stn{up, dn, mask, valid};
}

// Rules R1 (steepest neighbours) and R2 (saddle links) at one vertex.
template <int EM>
__device__ __forceinline__ void check_vertex(const Dev &D, EmitQ &q, const uint32_t *smulti,
                                             const int64_t *sdl, uint32_t fid, uint64_t vbase,
                                             uint32_t N, uint64_t i, uint32_t d, Stn g)
{
    const uint32_t upf = d & 15u, dnf = (d >> 4) & 15u, mf = (d >> 8) & 0x3FFFu;
    if (g.up != upf) emit<EM>(D, q, fid, vbase, N, (uint64_t)((int64_t)i + sdl[g.up]));
    if (g.dn != dnf) emit<EM>(D, q, fid, vbase, N, (uint64_t)((int64_t)i + sdl[dnf]));
    uint32_t diff = g.mask ^ mf;
    if (diff && ((d & D_SADDLE) || is_saddle(smulti, g.mask, g.valid))) {
        bool self = false;
        while (diff) {
            int s = __ffs(diff) - 1;
            diff &= diff - 1;
            if ((mf >> s) & 1u) emit<EM>(D, q, fid, vbase, N, (uint64_t)((int64_t)i + sdl[rank_of(s)]));
            else self = true;
        }
        if (self) emit<EM>(D, q, fid, vbase, N, i);
    }
}

template <int MODE>
__global__ void __launch_bounds__(CTA) k_stencil(Dev D, uint32_t *desc_out, uint8_t *type_out)
{
    __shared__ float sa[HALO_N];
    __shared__ float sb[MODE == SM_SETUP ? HALO_N : 1];
    __shared__ uint32_t smulti[512];
    __shared__ int64_t sdl[15];
    __shared__ EmitQ q;
    __shared__ uint32_t s_err;

    for (int j = threadIdx.x; j < 512; j += CTA) smulti[j] = D.multi[j];
    if (threadIdx.x == 0) {
        q.n = 0;
        s_err = 0;
    }
    unsigned long long count;
    const uint32_t *list = nullptr;
    if (MODE == SM_SETUP || MODE == SM_CHECK_ALL || MODE == SM_CLASSIFY) {
        count = D.total_tiles;
    } else if (MODE == SM_CHECK_LIST) {
        uint32_t c = D.ls->cur;
        count = D.ls->tile_count[c];
        list = D.tile_list[c];
    } else {
        count = D.ls->pin_tile_count;
        list = D.pin_tile_list;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int EM = MODE == SM_SETUP ? EM_FIRST : (MODE == SM_PINNED ? EM_PINNED : EM_NORMAL);

    for (unsigned long long it = blockIdx.x; it < count; it += gridDim.x) {
        const uint32_t tile = list ? list[it] : (uint32_t)it;
        const uint32_t fid = field_of_tile(D, tile);
        const FieldDesc &F = D.fields[fid];
        const uint64_t nx = F.nx, ny = F.ny, nz = F.nz, nxny = nx * ny;
        const uint64_t vbase = F.vbase;
        const uint32_t N = F.N;
        const uint64_t lt = tile - F.tbase;
        const uint32_t tx = (uint32_t)(lt % F.tnx);
        const uint64_t rest = lt / F.tnx;
        const uint32_t ty = (uint32_t)(rest % F.tny), tz = (uint32_t)(rest / F.tny);
        const int64_t x0 = (int64_t)tx * TX, y0 = (int64_t)ty * TY, z0 = (int64_t)tz * TZ;
        if (MODE == SM_CHECK_LIST && threadIdx.x == 0)
            atomicAnd(&D.tile_bits[tile >> 5], ~(1u << (tile & 31)));
        if (threadIdx.x < 15) sdl[threadIdx.x] = lin_delta(threadIdx.x, nx, nxny);

        const float *A = (MODE == SM_SETUP || MODE == SM_CLASSIFY) ? F.f : F.g;
        for (int j = threadIdx.x; j < HALO_N; j += CTA) {
            const int hx = j % HXP, r2 = j / HXP, hy = r2 % HY, hz = r2 / HY;
            const int64_t X = x0 - 1 + hx, Y = y0 - 1 + hy, Z = z0 - 1 + hz;
            const bool in = X >= 0 && Y >= 0 && Z >= 0 && X < (int64_t)nx && Y < (int64_t)ny &&
                            Z < (int64_t)nz;
            const uint64_t idx = (uint64_t)X + nx * ((uint64_t)Y + ny * (uint64_t)Z);
            sa[j] = in ? A[idx] : __int_as_float(0x7fc00000);
            if (MODE == SM_SETUP) sb[j] = in ? F.fhat[idx] : __int_as_float(0x7fc00000);
        }
        __syncthreads();
        const bool interior = x0 >= 1 && x0 + TX < (int64_t)nx && y0 >= 1 && y0 + TY < (int64_t)ny &&
                              z0 >= 1 && z0 + TZ < (int64_t)nz;

        for (int rr = warp; rr < ROWS; rr += WARPS) {
            const int ly = rr % TY, lz = rr / TY;
            const uint64_t x = (uint64_t)(x0 + lane), y = (uint64_t)(y0 + ly), z = (uint64_t)(z0 + lz);
            const bool in = x < nx && y < ny && z < nz;
            const int c = ((lz + 1) * HY + (ly + 1)) * HXP + (lane + 1);
            bool cp = false;
            if (in) {
                const uint64_t i = x + nx * (y + ny * z);
                if (MODE == SM_SETUP || MODE == SM_CLASSIFY) {
                    Stn sf = interior ? stencil15<true>(sa, c) : stencil15<false>(sa, c);
                    const uint32_t L = sf.mask, U = sf.valid & ~sf.mask;
                    const bool mn = L == 0, mxx = !mn && U == 0;
                    const bool join = !mn && !mxx && multi_bit(smulti, L);
                    const bool split = !mn && !mxx && multi_bit(smulti, U);
                    cp = mn || mxx || join || split;
                    const uint32_t d = sf.up | (sf.dn << 4) | (sf.mask << 8) |
                                       ((join || split) ? D_SADDLE : 0u) | (cp ? D_CP : 0u);
                    if (MODE == SM_CLASSIFY) {
                        desc_out[i] = d;
                        if (type_out)
                            type_out[i] = (uint8_t)(mn ? 1 : (mxx ? 2 : ((join ? 4 : 0) | (split ? 8 : 0))));
                    } else {
                        const float fv = sa[c], hv = sb[c];
                        uint32_t e = 0;
                        if (!isfinite(fv) || !isfinite(hv)) e = ERR_NONFINITE;
                        else if (hv < __fsub_rn(fv, F.xi) || hv > __fadd_rn(fv, F.xi)) e = ERR_BOUND;
                        if (e) atomicOr(&s_err, e);
                        D.desc[vbase + i] = d;
                        D.k[vbase + i] = 0;
                        F.g[i] = hv;
                        Stn sg = interior ? stencil15<true>(sb, c) : stencil15<false>(sb, c);
                        check_vertex<EM>(D, q, smulti, sdl, fid, vbase, N, i, d, sg);
                    }
                } else {
                    const uint32_t d = __ldg(&D.desc[vbase + i]);
                    Stn sg = interior ? stencil15<true>(sa, c) : stencil15<false>(sa, c);
                    check_vertex<EM>(D, q, smulti, sdl, fid, vbase, N, i, d, sg);
                }
            }
            if (MODE == SM_SETUP) {
                const uint32_t w = __ballot_sync(0xffffffffu, cp);
                if (lane == 0 && y < ny && z < nz) D.cpwords[F.wbase + (z * ny + y) * F.tnx + tx] = w;
            }
        }
        if (MODE != SM_CLASSIFY) q_flush(q, D);
        else __syncthreads();
        if (MODE == SM_SETUP && threadIdx.x == 0 && s_err) {
            atomicOr(&D.fst[fid].err, s_err);
            s_err = 0;
        }
    }
}

// ------------------------------------------------------------ block scan helpers
// Exclusive scan of one uint32 per thread across the block; returns the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t &excl, uint32_t *swarp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) swarp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < WARPS ? swarp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < WARPS) swarp[lane] = w;
    }
    __syncthreads();
    const uint32_t before = warp ? swarp[warp - 1] : 0;
    const uint32_t total = swarp[WARPS - 1];
    excl = before + x - v;
    __syncthreads();
    return total;
}

// Exclusive scan of n uint32 values into uint64 offsets; one block of 1024.
__global__ void __launch_bounds__(1024) k_scan_u32(const uint32_t *in, unsigned long long *out, uint64_t n,
                                                   unsigned long long *total)
{
    __shared__ unsigned long long sw[32];
    const uint64_t per = (n + 1023) / 1024;
    const uint64_t b = threadIdx.x * per, e = min(n, b + per);
    unsigned long long s = 0;
    for (uint64_t j = b; j < e; j++) s += in[j];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = s;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = sw[lane];
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sw[lane] = w;
    }
    __syncthreads();
    unsigned long long run = (warp ? sw[warp - 1] : 0) + x - s;
    for (uint64_t j = b; j < e; j++) {
        out[j] = run;
        run += in[j];
    }
    if (threadIdx.x == 1023 && total) *total = sw[31];
}

// In-place exclusive scan of n uint32 values (sum < 2^32); one block of 1024.
__global__ void __launch_bounds__(1024) k_scan_inplace_u32(uint32_t *a, uint64_t n)
{
    __shared__ uint32_t sw[32];
    const uint64_t per = (n + 1023) / 1024;
    const uint64_t b = threadIdx.x * per, e = min(n, b + per);
    uint32_t s = 0;
    for (uint64_t j = b; j < e; j++) s += a[j];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = sw[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sw[lane] = w;
    }
    __syncthreads();
    uint32_t run = (warp ? sw[warp - 1] : 0) + x - s;
    for (uint64_t j = b; j < e; j++) {
        uint32_t v = a[j];
        a[j] = run;
        run += v;
    }
}

// ------------------------------------------------------------ CP compaction
constexpr int WPT = WBLOCK / CTA;  // cp-bitmap words per thread

__device__ __forceinline__ uint32_t field_of_word(const Dev &D, uint64_t w)
{
    uint32_t lo = 0, hi = D.nfields - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (D.fields[mid].wbase <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(CTA) k_cp_count(Dev D)
{
    __shared__ uint32_t sw[WARPS];
    const uint64_t w0 = (uint64_t)blockIdx.x * WBLOCK + threadIdx.x * WPT;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < WPT; j++) c += __popc(D.cpwords[w0 + j]);
    uint32_t ex;
    uint32_t tot = block_excl_scan(c, ex, sw);
    if (threadIdx.x == 0) D.blk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(CTA) k_cp_write(Dev D)
{
    __shared__ uint32_t sw[WARPS];
    const uint64_t blk0 = (uint64_t)blockIdx.x * WBLOCK;
    const uint32_t fid = field_of_word(D, blk0);
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
    block_excl_scan(c, ex, sw);
    unsigned long long pos = D.blk_off[blockIdx.x] + ex;
    if (blk0 == F.wbase && threadIdx.x == 0) D.fst[fid].cp_base = D.blk_off[blockIdx.x];
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

__global__ void k_cp_ncp(Dev D)
{
    const unsigned long long total = D.ls->total_cp;
    for (uint32_t f = threadIdx.x + blockIdx.x * blockDim.x; f < D.nfields; f += blockDim.x * gridDim.x) {
        const unsigned long long b = D.fst[f].cp_base;
        const unsigned long long e = (f + 1 < D.nfields) ? D.fst[f + 1].cp_base : total;
        D.fst[f].ncp = e - b;
    }
}

// ------------------------------------------------------------ radix sort (stable LSD)
// Pass p < 4: digit p of the 32-bit value key; pass p >= 4: digit p-4 of the field id.
__device__ __forceinline__ uint32_t sort_digit(int pass, uint32_t key, unsigned long long ent)
{
    if (pass < 4) return (key >> (8 * pass)) & 255u;
    return (uint32_t)(ent >> (LOCAL_BITS + 8 * (pass - 4))) & 255u;
}

__global__ void __launch_bounds__(CTA) k_sort_hist(Dev D, int pass, const uint32_t *ksrc,
                                                   const unsigned long long *esrc)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const unsigned long long count = D.ls->total_cp;
    const unsigned long long chunk = (count + gridDim.x - 1) / gridDim.x;
    const unsigned long long b = blockIdx.x * chunk, e = min(count, b + chunk);
    for (unsigned long long j = b + threadIdx.x; j < e; j += CTA) {
        const uint32_t key = pass < 4 ? ksrc[j] : 0u;
        const unsigned long long ent = pass < 4 ? 0ull : esrc[j];
        atomicAdd(&h[sort_digit(pass, key, ent)], 1u);
    }
    __syncthreads();
    D.hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(CTA) k_sort_scatter(Dev D, int pass, const uint32_t *ksrc,
                                                      const unsigned long long *esrc, uint32_t *kdst,
                                                      unsigned long long *edst)
{
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_wc[WARPS][256];
    __shared__ uint32_t s_tot[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long count = D.ls->total_cp;
    const unsigned long long chunk = (count + gridDim.x - 1) / gridDim.x;
    const unsigned long long b = blockIdx.x * chunk, e = min(count, b + chunk);
    s_run[threadIdx.x] = D.hist[threadIdx.x * gridDim.x + blockIdx.x];
    const bool move_keys = pass < 3;  // keys are not needed after the last value pass
    for (unsigned long long base = b; base < e; base += CTA) {
#pragma unroll
        for (int w = 0; w < WARPS; w++) s_wc[w][threadIdx.x] = 0;
        __syncthreads();
        const unsigned long long j = base + threadIdx.x;
        const bool valid = j < e;
        uint32_t key = 0;
        unsigned long long ent = 0;
        uint32_t d = 0x100u + 0;  // never equals a real digit
        if (valid) {
            if (pass < 4) key = ksrc[j];
            ent = esrc[j];
            d = sort_digit(pass, key, ent);
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < WARPS; w++) {
                const uint32_t t = s_wc[w][threadIdx.x];
                s_wc[w][threadIdx.x] = s;
                s += t;
            }
            s_tot[threadIdx.x] = s;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_run[d] + s_wc[warp][d] + rank;
            if (move_keys) kdst[pos] = key;
            edst[pos] = ent;
        }
        __syncthreads();
        s_run[threadIdx.x] += s_tot[threadIdx.x];
        __syncthreads();
    }
}

__global__ void k_cp_rank(Dev D)
{
    const unsigned long long total = D.ls->total_cp;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < total;
         q += (unsigned long long)blockDim.x * gridDim.x) {
        const unsigned long long e = D.o[q];
        const uint32_t fid = (uint32_t)(e >> LOCAL_BITS);
        const FieldDesc &F = D.fields[fid];
        D.cp_rank[F.vbase + (e & LOCAL_MASK)] = (uint32_t)(q - D.fst[fid].cp_base);
    }
}

// ------------------------------------------------------------ pair check (Sec. 4.3)
enum { PM_ALL = 0, PM_LIST = 1, PM_PINNED = 2 };

__device__ __forceinline__ void warp_push(const Dev &D, bool has, unsigned long long e)
{
    const uint32_t m = __ballot_sync(0xffffffffu, has);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&D.ls->req_count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (has) D.req_list[base + __popc(m & lanemask_lt())] = e;
}

template <int PM>
__global__ void __launch_bounds__(CTA) k_pairs(Dev D)
{
    const unsigned long long total = D.ls->total_cp;
    unsigned long long count;
    const uint32_t *list = nullptr;
    if (PM == PM_ALL) {
        count = total ? total - 1 : 0;
    } else if (PM == PM_LIST) {
        const uint32_t c = D.ls->cur;
        count = D.ls->pair_count[c];
        list = D.pair_list[c];
    } else {
        count = D.ls->pin_pair_count;
        list = D.pin_pair_list;
    }
    const unsigned long long stride = (unsigned long long)gridDim.x * CTA;
    for (unsigned long long base = (unsigned long long)blockIdx.x * CTA; base < count; base += stride) {
        const unsigned long long j = base + threadIdx.x;
        bool has = false;
        unsigned long long e = 0;
        if (j < count) {
            const unsigned long long q = list ? list[j] : j;
            if (q + 1 < total) {
                const unsigned long long a = D.o[q], b = D.o[q + 1];
                if ((a >> LOCAL_BITS) == (b >> LOCAL_BITS)) {
                    const uint32_t fid = (uint32_t)(a >> LOCAL_BITS);
                    const FieldDesc &F = D.fields[fid];
                    const uint64_t la = a & LOCAL_MASK, lb = b & LOCAL_MASK;
                    const float ga = F.g[la], gb = F.g[lb];
                    if (gb < ga || (gb == ga && lb < la)) {
                        const uint64_t gid = F.vbase + la;
                        const uint8_t kk = D.k[gid];
                        const bool ok = PM == PM_PINNED ? (kk > F.N) : (kk <= F.N);
                        if (ok) {
                            const uint32_t bit = 1u << (gid & 31);
                            uint32_t *w = &D.reqbits[gid >> 5];
                            if (!(__ldcg(w) & bit) && !(atomicOr(w, bit) & bit)) {
                                has = true;
                                e = a;
                            }
                        }
                    }
                }
            }
        }
        warp_push(D, has, e);
    }
}

// ------------------------------------------------------------ apply (Sec. 3.3)
__device__ __forceinline__ void mark_star_tiles(const Dev &D, const FieldDesc &F, uint64_t t, uint32_t *bits,
                                                uint32_t *list, unsigned long long *count)
{
    const uint64_t nx = F.nx, ny = F.ny, nz = F.nz;
    const int64_t x = (int64_t)(t % nx), y = (int64_t)((t / nx) % ny), z = (int64_t)(t / (nx * ny));
    uint32_t seen[8];
    int ns = 0;
#pragma unroll 1
    for (int r = 0; r < 15; r++) {
        const int64_t X = x + rdx(r), Y = y + rdy(r), Z = z + rdz(r);
        if (X < 0 || Y < 0 || Z < 0 || X >= (int64_t)nx || Y >= (int64_t)ny || Z >= (int64_t)nz) continue;
        const uint32_t tile = (uint32_t)(F.tbase + (uint64_t)(X / TX) +
                                         (uint64_t)F.tnx * ((uint64_t)(Y / TY) + (uint64_t)F.tny * (uint64_t)(Z / TZ)));
        bool dup = false;
        for (int s = 0; s < ns; s++) dup |= seen[s] == tile;
        if (dup) continue;
        if (ns < 8) seen[ns++] = tile;
        mark_tile(bits, list, count, tile);
    }
}

__global__ void __launch_bounds__(CTA) k_apply(Dev D, int frontier)
{
    const unsigned long long count = D.ls->req_count;
    const uint32_t nxt = D.ls->cur ^ 1u;
    for (unsigned long long j = blockIdx.x * (unsigned long long)CTA + threadIdx.x; j < count;
         j += (unsigned long long)gridDim.x * CTA) {
        const unsigned long long e = D.req_list[j];
        const uint32_t fid = (uint32_t)(e >> LOCAL_BITS);
        const uint64_t t = e & LOCAL_MASK;
        const FieldDesc &F = D.fields[fid];
        FieldState *S = &D.fst[fid];
        const uint64_t gid = F.vbase + t;
        atomicAnd(&D.reqbits[gid >> 5], ~(1u << (gid & 31)));
        if (S->err) continue;
        if (S->iterations >= F.max_iters) {
            atomicAdd(&S->capped, 1ull);
            continue;
        }
        const uint32_t N = F.N;
        uint32_t kk = D.k[gid];
        if (kk > N) continue;
        const float fl = __fsub_rn(F.f[t], F.xi);
        float gv;
        if (kk < N) {
            const float tt = __fsub_rn(F.g[t], F.delta);
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
        F.g[t] = gv;
        D.k[gid] = (uint8_t)kk;
        S->had_req = 1;
        const bool pinned = kk == N + 1;
        if (frontier) mark_star_tiles(D, F, t, D.tile_bits, D.tile_list[nxt], &D.ls->tile_count[nxt]);
        if (pinned) mark_star_tiles(D, F, t, D.pin_tile_bits, D.pin_tile_list, &D.ls->pin_tile_count);
        if ((frontier || pinned) && (D.desc[gid] & D_CP)) {
            const unsigned long long q = S->cp_base + D.cp_rank[gid];
            const unsigned long long r = D.cp_rank[gid];
            const int np = (r >= 1) ? 2 : 1;
            if (frontier) {
                const unsigned long long p = atomicAdd(&D.ls->pair_count[nxt], (unsigned long long)np);
                D.pair_list[nxt][p] = (uint32_t)q;
                if (np == 2) D.pair_list[nxt][p + 1] = (uint32_t)(q - 1);
            }
            if (pinned) {
                const unsigned long long p = atomicAdd(&D.ls->pin_pair_count, (unsigned long long)np);
                D.pin_pair_list[p] = (uint32_t)q;
                if (np == 2) D.pin_pair_list[p + 1] = (uint32_t)(q - 1);
            }
        }
    }
}

// ------------------------------------------------------------ bookkeeping
__global__ void __launch_bounds__(CTA) k_book(Dev D, cudaGraphConditionalHandle h, int use_graph)
{
    __shared__ uint32_t s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (uint32_t f = threadIdx.x; f < D.nfields; f += CTA) {
        FieldState *S = &D.fst[f];
        if (S->done) continue;
        if (S->err || S->capped) {
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
        const uint32_t c = L->cur;
        L->tile_count[c] = 0;
        L->pair_count[c] = 0;
        L->cur = c ^ 1u;
        L->req_count = 0;
        L->pass += 1;
        L->any_active = s_any;
        if (use_graph) cudaGraphSetConditional(h, s_any ? 1u : 0u);
    }
}

// Sets the loop flag (and graph conditional) from the per-field state.
__global__ void k_loop_flag(Dev D, cudaGraphConditionalHandle h, int use_graph)
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

// ------------------------------------------------------------ residual / status
__global__ void __launch_bounds__(CTA) k_finish(Dev D)
{
    const unsigned long long count = D.ls->req_count;
    for (unsigned long long j = blockIdx.x * (unsigned long long)CTA + threadIdx.x; j < count;
         j += (unsigned long long)gridDim.x * CTA) {
        const unsigned long long e = D.req_list[j];
        const uint32_t fid = (uint32_t)(e >> LOCAL_BITS);
        const uint64_t gid = D.fields[fid].vbase + (e & LOCAL_MASK);
        atomicAnd(&D.reqbits[gid >> 5], ~(1u << (gid & 31)));
        atomicAdd(&D.fst[fid].pinned_res, 1ull);
    }
}

__global__ void k_status(Dev D)
{
    for (uint32_t f = threadIdx.x + blockIdx.x * blockDim.x; f < D.nfields; f += blockDim.x * gridDim.x) {
        FieldState *S = &D.fst[f];
        if (S->err & ERR_NONFINITE) S->status = (uint32_t)-2;
        else if (S->err & ERR_BOUND) S->status = (uint32_t)-3;
        else if (S->capped) S->status = ST_ITER_LIMIT;
        else S->status = (S->pinned_res ? ST_STUCK : ST_CONVERGED);
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) D.ls->req_count = 0;
}

// ------------------------------------------------------------ edit list
constexpr int EPT = VBLOCK / CTA;  // arena vertices per thread

__device__ __forceinline__ uint32_t field_of_vertex(const Dev &D, uint64_t v)
{
    uint32_t lo = 0, hi = D.nfields - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (D.fields[mid].vbase <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(CTA) k_edit_count(Dev D)
{
    __shared__ uint32_t sw[WARPS];
    __shared__ uint32_t s_lossless;
    if (threadIdx.x == 0) s_lossless = 0;
    const uint64_t v0 = (uint64_t)blockIdx.x * VBLOCK;
    const uint32_t fid = field_of_vertex(D, v0);
    const uint32_t N = D.fields[fid].N;
    const uint64_t b = v0 + threadIdx.x * EPT;
    uint32_t c = 0, l = 0;
    const uint4 *kp = reinterpret_cast<const uint4 *>(D.k + b);
    for (int j = 0; j < EPT / 16; j++) {
        const uint4 w = kp[j];
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int u = 0; u < 4; u++) {
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const uint32_t kk = (ws[u] >> (8 * s)) & 255u;
                c += kk != 0;
                l += kk == N + 1;
            }
        }
    }
    __syncthreads();
    if (l) atomicAdd(&s_lossless, l);
    uint32_t ex;
    const uint32_t tot = block_excl_scan(c, ex, sw);
    if (threadIdx.x == 0) {
        D.blk[blockIdx.x] = tot;
        if (tot) atomicAdd(&D.fst[fid].n_edits, (unsigned long long)tot);
        if (s_lossless) atomicAdd(&D.fst[fid].n_lossless, (unsigned long long)s_lossless);
    }
}

__global__ void __launch_bounds__(CTA) k_edit_write(Dev D)
{
    __shared__ uint32_t sw[WARPS];
    const uint64_t v0 = (uint64_t)blockIdx.x * VBLOCK;
    const uint32_t fid = field_of_vertex(D, v0);
    const FieldDesc &F = D.fields[fid];
    if (!F.edits) return;
    const uint32_t N = F.N;
    const uint64_t b = v0 + threadIdx.x * EPT;
    uint32_t c = 0;
    for (int j = 0; j < EPT; j++) c += D.k[b + j] != 0;
    uint32_t ex;
    block_excl_scan(c, ex, sw);
    const unsigned long long fbase = D.blk_off[F.vbase / VBLOCK];
    unsigned long long pos = D.blk_off[blockIdx.x] + ex - fbase;
    if (!c) return;
    for (int j = 0; j < EPT; j++) {
        const uint32_t kk = D.k[b + j];
        if (!kk) continue;
        if (pos < F.edits_cap) {
            const uint64_t t = b + j - F.vbase;
            EditRec r;
            r.idx = t;
            r.value = F.g[t];
            r.k = (uint8_t)kk;
            r.lossless = kk == N + 1;
            r.reserved = 0;
            F.edits[pos] = r;
        }
        pos++;
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

void launch_setup(const Dev &D, cudaStream_t s)
{
    k_stencil<SM_SETUP><<<grid_for(D.total_tiles, 1, 16), CTA, 0, s>>>(D, nullptr, nullptr);
}
void launch_check_all(const Dev &D, cudaStream_t s)
{
    k_stencil<SM_CHECK_ALL><<<grid_for(D.total_tiles, 1, 16), CTA, 0, s>>>(D, nullptr, nullptr);
}
void launch_check_list(const Dev &D, cudaStream_t s)
{
    k_stencil<SM_CHECK_LIST><<<grid_for(D.total_tiles, 1, 16), CTA, 0, s>>>(D, nullptr, nullptr);
}
void launch_check_pinned(const Dev &D, cudaStream_t s)
{
    k_stencil<SM_PINNED><<<grid_for(D.total_tiles, 1, 16), CTA, 0, s>>>(D, nullptr, nullptr);
}
void launch_classify(const Dev &D, uint32_t *desc_out, uint8_t *type_out, cudaStream_t s)
{
    k_stencil<SM_CLASSIFY><<<grid_for(D.total_tiles, 1, 16), CTA, 0, s>>>(D, desc_out, type_out);
}

void launch_cp_compact(const Dev &D, cudaStream_t s)
{
    const uint64_t nb = D.total_w / WBLOCK;
    k_cp_count<<<(unsigned)nb, CTA, 0, s>>>(D);
    k_scan_u32<<<1, 1024, 0, s>>>(D.blk, D.blk_off, nb, &D.ls->total_cp);
    k_cp_write<<<(unsigned)nb, CTA, 0, s>>>(D);
    k_cp_ncp<<<(D.nfields + 255) / 256, 256, 0, s>>>(D);
}

int sort_passes(uint32_t nfields)
{
    int p = 4;
    if (nfields > 1) p += 1;
    if (nfields > 256) p += 1;
    if (nfields > 65536) p += 1;
    return p;
}

void launch_cp_sort(const Dev &D, cudaStream_t s)
{
    const int P = sort_passes(D.nfields);
    const unsigned B = D.sort_blocks;
    int src = 0;
    for (int p = 0; p < P; p++) {
        const int dst = src ^ 1;
        k_sort_hist<<<B, CTA, 0, s>>>(D, p, D.cp_key[src], D.cp_ent[src]);
        k_scan_inplace_u32<<<1, 1024, 0, s>>>(D.hist, (uint64_t)256 * B);
        k_sort_scatter<<<B, CTA, 0, s>>>(D, p, D.cp_key[src], D.cp_ent[src], D.cp_key[dst], D.cp_ent[dst]);
        src = dst;
    }
    k_cp_rank<<<sms() * 8, 256, 0, s>>>(D);
}

void launch_pairs_all(const Dev &D, cudaStream_t s) { k_pairs<PM_ALL><<<sms() * 8, CTA, 0, s>>>(D); }
void launch_pairs_list(const Dev &D, cudaStream_t s) { k_pairs<PM_LIST><<<sms() * 4, CTA, 0, s>>>(D); }
void launch_pairs_pinned(const Dev &D, cudaStream_t s) { k_pairs<PM_PINNED><<<sms() * 2, CTA, 0, s>>>(D); }

void launch_apply(const Dev &D, int frontier, cudaStream_t s)
{
    k_apply<<<sms() * 8, CTA, 0, s>>>(D, frontier);
}
void launch_book(const Dev &D, cudaGraphConditionalHandle h, int use_graph, cudaStream_t s)
{
    k_book<<<1, CTA, 0, s>>>(D, h, use_graph);
}
void launch_loop_flag(const Dev &D, cudaGraphConditionalHandle h, int use_graph, cudaStream_t s)
{
    k_loop_flag<<<1, 256, 0, s>>>(D, h, use_graph);
}
void launch_finish(const Dev &D, cudaStream_t s)
{
    k_finish<<<sms() * 2, CTA, 0, s>>>(D);
    k_status<<<(D.nfields + 255) / 256, 256, 0, s>>>(D);
}
void launch_edit_list(const Dev &D, int write, cudaStream_t s)
{
    const uint64_t nb = D.total_v / VBLOCK;
    k_edit_count<<<(unsigned)nb, CTA, 0, s>>>(D);
    if (write) {
        k_scan_u32<<<1, 1024, 0, s>>>(D.blk, D.blk_off, nb, nullptr);
        k_edit_write<<<(unsigned)nb, CTA, 0, s>>>(D);
    }
}

}  // namespace exz
