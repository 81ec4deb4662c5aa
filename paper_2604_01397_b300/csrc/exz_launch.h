// exz_launch.h -- host-side launchers of the kernels in exz_kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "exz_common.cuh"

namespace exz {

void launch_fill_u32(uint32_t *p, uint32_t v, uint64_t n, cudaStream_t s);
// cudaMalloc through the library's allocation-failure injection (a testing aid,
// exactz_debug_fail_allocations): an injected failure returns
// cudaErrorMemoryAllocation without calling cudaMalloc.
cudaError_t dev_malloc_bytes(void **p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc_bytes(reinterpret_cast<void **>(p), bytes);
}
int device_sms();
// 2^14-bit link-component table (host copy, built on first use; see exz_engine.cu)
const uint32_t *host_multi_table();
// TMA map of a field's halo box (halo) or descriptor tile; false where the field cannot be mapped
// (pitch: row pitch of the array in elements, 0 for nx)
bool make_map(CUtensorMap *map, const void *base, const FieldDesc &F, bool halo, uint32_t pitch = 0);

void launch_setup(const Dev &D, const SetupRange &R, cudaStream_t s);
void launch_check_all(const Dev &D, cudaStream_t s);
void launch_check_list(const Dev &D, cudaStream_t s);
void launch_check_pinned(const Dev &D, const FieldSet &FS, cudaStream_t s);
void launch_classify(const Dev &D, uint32_t *desc_out, uint8_t *type_out, cudaStream_t s);
void launch_cp_compact(const Dev &D, const SetupRange &R, cudaStream_t s);
void launch_cp_sort(const Dev &D, const SetupRange &R, cudaStream_t s);
int sort_passes(uint32_t fid0, uint32_t fid1);
void launch_pairs_all(const Dev &D, const SetupRange &R, cudaStream_t s);
void launch_pairs_list(const Dev &D, cudaStream_t s);
void launch_pairs_pinned(const Dev &D, const FieldSet &FS, cudaStream_t s);
void launch_apply(const Dev &D, int frontier, cudaStream_t s);
// event lists of the original event constraints (set-up)
void launch_ev_init(const Dev &D, uint32_t *E, cudaStream_t s);
void launch_ev_jump(const Dev &D, uint32_t *E, uint8_t *tdone, cudaStream_t s);
void launch_ev_lists(const Dev &D, const uint32_t *E, int write, uint32_t *room,
                     const unsigned long long *room_off, uint32_t *list, uint32_t *start, uint16_t *cnt,
                     cudaStream_t s);
// exclusive scan of n uint32 into uint64 offsets (one block), *total = the sum (may be null)
void launch_scan_u32(const uint32_t *in, unsigned long long *out, uint64_t n, unsigned long long *total,
                     cudaStream_t s);
void launch_ev_reverse(const Dev &D, uint32_t *radj, cudaStream_t s);
void launch_book(const Dev &D, cudaGraphConditionalHandle h, int use_graph, cudaStream_t s);
// One frontier pass (check, CP pairs, apply, bookkeeping) as one cooperative kernel launch of
// pass_grid() blocks: as many as can be resident at once.
cudaError_t pass_grid(unsigned *grid);
cudaError_t launch_pass(const Dev &D, cudaGraphConditionalHandle h, unsigned grid, cudaStream_t s);
void launch_loop_flag(const Dev &D, cudaGraphConditionalHandle h, int use_graph, cudaStream_t s);
void launch_finish(const Dev &D, const FieldSet &FS, cudaStream_t s);
void launch_edit_list(const Dev &D, const FieldSet &FS, int write, cudaStream_t s);
// increasing edits by reflection of the field
void launch_reflect_in(const float *src, float *dst, uint64_t n, cudaStream_t s);
void launch_reflect_out(float *g, const uint32_t *desc, uint64_t n, cudaStream_t s);
// g of the fields kept in a padded copy (FieldDesc::gm) copied back into FieldDesc::g.
void launch_unmirror(const Dev &D, cudaStream_t s);
// edit stream (storage form of a result)
unsigned stream_blocks(uint64_t items);
void launch_stream_kcodes(const EditRec *edits, uint64_t ne, uint64_t n, uint32_t N, uint8_t *kcodes, int *bad,
                          cudaStream_t s);
void launch_stream_count(const EditRec *edits, const uint8_t *kcodes, uint64_t n, uint32_t N, int from_codes,
                         uint32_t *blk, int *bad, cudaStream_t s);
void launch_stream_lossless(const EditRec *edits, uint64_t ne, const unsigned long long *blk_off, float *lossless,
                            cudaStream_t s);
void launch_stream_decode(const float *fhat, const uint8_t *kcodes, const float *lossless, uint64_t n, uint32_t N,
                          float delta, int inc, const unsigned long long *blk_off, float *g, cudaStream_t s);

}  // namespace exz
