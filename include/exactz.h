/*
 * exactz.h -- C ABI of the B300 (sm_103a) EXaCTz topology correction.
 *
 * The operation (Li et al., EXaCTz, Sec. 4.1 problem statement and Algorithm 1):
 * given an original float32 scalar field f on a regular grid, an error-bounded
 * decompressed version f_hat with |f_hat - f| <= xi, and the bound xi, edit
 * f_hat by monotone decreasing steps of Delta = xi / N (Sec. 3.3) until, on the
 * Freudenthal triangulation of the grid with ties broken by vertex index
 * (Sec. 3.3 footnote):
 *   - every vertex has the same steepest-ascent and steepest-descent vertex in
 *     its closed neighbourhood as in f (EG constraints, Sec. 4.2);
 *   - every vertex that is a saddle of f or of the edited field orders against
 *     all its neighbours as in f (Sec. 4.2, saddles);
 *   - all critical points of f keep f's global order (reformulated event
 *     constraints, Sec. 4.3, which subsume the saddle-ordering constraint C2);
 *     or, with opts.events = EXACTZ_EVENTS_ORIGINAL, the saddles of f keep
 *     their order (C2) and every saddle keeps the extremum that Extremum Graph
 *     Pairing selects among the extrema its integral paths reach in f (merge
 *     and split event constraints C3, Sec. 4.2).
 * A vertex needing more than N edits stores the lossless bound fl(f - xi).
 * The result is the edited field g, the sparse edit list and the number of
 * edit passes; at the fixpoint the extremum graphs and the contour tree of g
 * equal those of f.
 *
 * Layout: a field of dims (nx, ny, nz) is nx*ny*nz float32 values with x
 * fastest: vertex index = x + nx * (y + ny * z).  nz = 1 gives a 2D field,
 * ny = nz = 1 a 1D field.  Every dimension must be >= 1 and the field must hold
 * at least 2 vertices and fewer than 2^40.
 *
 * Memory: unless a call says otherwise, every array pointer is a DEVICE pointer
 * owned by the caller (for example a torch CUDA tensor's data pointer).  The
 * library never frees caller memory.  It allocates its own device workspace
 * (about 40-70 bytes per vertex, depending on the number of critical points):
 * exactz_correct / exactz_correct_batch allocate and free it inside the call;
 * an exactz_workspace keeps it across calls.
 *
 * Streams: `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 * Every call is synchronous with respect to that stream on return: the
 * results are in device memory and the result structs are filled.  There is
 * no CPU fallback: without a usable CUDA device every call returns
 * EXACTZ_ENODEV.
 */
#ifndef EXACTZ_H
#define EXACTZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes (negative = error, the call did not produce a result). */
#define EXACTZ_OK 0
#define EXACTZ_EINVAL (-1)     /* bad dims, xi <= 0 or non-finite, N out of [1, 254], NULL pointer */
#define EXACTZ_ENONFINITE (-2) /* NaN or Inf in f or f_hat */
#define EXACTZ_EBOUND (-3)     /* some f_hat_i < fl(f_i - xi) or f_hat_i > fl(f_i + xi) */
#define EXACTZ_ENOMEM (-4)     /* device allocation failed */
#define EXACTZ_ECAP (-5)       /* edit list longer than edits_cap: first edits_cap records written */
#define EXACTZ_ENODEV (-6)     /* no CUDA device / CUDA error */
#define EXACTZ_ESIZE (-7)      /* workspace too small for these fields */

/* Positive outcome codes in exactz_result.status. */
#define EXACTZ_CONVERGED 1   /* no constraint is violated */
#define EXACTZ_STUCK 2       /* violations remain only on vertices already at fl(f - xi) */
#define EXACTZ_ITER_LIMIT 3  /* opts.max_iters edit passes done, violations remain */

/* Iteration strategies (opts.mode). */
#define EXACTZ_MODE_PLAIN 0     /* Algorithm 1 literally: full sweep each pass, host-driven loop */
#define EXACTZ_MODE_FRONTIER 1  /* re-check only tiles touched by last pass's edits, host-driven loop */
#define EXACTZ_MODE_GRAPH 2     /* frontier passes in a CUDA graph; device-side while-loop exit */
#define EXACTZ_MODE_FUSED 3     /* the graph loop with each pass as one cooperatively launched kernel
                                 * (check and CP pairs, grid barrier, apply, bookkeeping); same results */

/* Edit direction (opts.direction).  Every rule names the vertex that must be
 * lower (decreasing edits, Sec. 3.3: g <- fl(g - Delta) down to fl(f - xi)) or
 * the one that must be higher (increasing edits: g <- fl(g + Delta) up to
 * fl(f + xi)); the paper's framework allows either and uses decreasing.  The
 * increasing correction is computed as the decreasing one of the point
 * reflection x -> (nx-1-x, ny-1-y, nz-1-z) of -f, -f_hat (which maps the mesh
 * onto itself and reverses the order with its index tie-break), mapped back;
 * it needs 8 bytes per vertex of extra workspace. */
#define EXACTZ_EDITS_DECREASING 0
#define EXACTZ_EDITS_INCREASING 1

/* Event constraints (opts.events). */
#define EXACTZ_EVENTS_REFORMULATED 0 /* global order of all critical points (Sec. 4.3) */
#define EXACTZ_EVENTS_ORIGINAL 1     /* saddle order C2 + extremum-graph merge/split events C3 (Sec. 4.2);
                                        set-up traces the integral paths of f once (pointer jumping);
                                        the workspace's fields below 2^31 vertices in all */

typedef struct {
    uint32_t nx, ny, nz;
} exactz_dims;

typedef struct {
    uint32_t N;              /* edit steps per vertex before the lossless bound (paper: 5) */
    uint32_t mode;           /* EXACTZ_MODE_* (default EXACTZ_MODE_GRAPH) */
    uint64_t max_iters;      /* cap on edit passes (0 = no edit is applied) */
    uint32_t want_edit_list; /* 0: skip the edit-list compaction */
    uint32_t profile;        /* 1: time the stages with CUDA events (see exactz_ws_stats) */
    uint32_t events;         /* EXACTZ_EVENTS_* (default REFORMULATED) */
    uint32_t direction;      /* EXACTZ_EDITS_* (default DECREASING) */
} exactz_opts;

/* One applied edit.  value = g at idx; k = number of decrements applied (1..N)
 * or N+1 for the lossless bound fl(f - xi) (lossless = 1).  16 bytes. */
typedef struct {
    uint64_t idx;
    float value;
    uint8_t k;
    uint8_t lossless;
    uint16_t reserved;
} exactz_edit;

typedef struct {
    uint64_t iterations;          /* edit passes executed */
    uint64_t n_edits;             /* vertices with k > 0 */
    uint64_t n_lossless;          /* vertices with k = N + 1 */
    uint64_t residual_violations; /* |request set| at exit (0 when converged) */
    uint64_t n_critical;          /* critical points of f */
    int32_t status;               /* EXACTZ_CONVERGED / _STUCK / _ITER_LIMIT, or a negative error */
    int32_t reserved;
} exactz_result;

/* Fill *o with the defaults: N = 5, mode = GRAPH, max_iters = 1000000,
 * want_edit_list = 1. */
void exactz_default_opts(exactz_opts *o);

/* Correct one field (Algorithm 1).  f, fhat, g_out: device arrays of n floats
 * (g_out may alias neither input).  edits_out: device array of edits_cap
 * records, or NULL with edits_cap = 0 (then only counts are returned).
 * opts may be NULL (defaults).  Returns EXACTZ_OK, EXACTZ_ECAP (result valid,
 * list truncated) or a negative error; res->status holds the outcome. */
int exactz_correct(const float *f, const float *fhat, exactz_dims d, float xi,
                   const exactz_opts *opts, float *g_out, exactz_edit *edits_out,
                   uint64_t edits_cap, exactz_result *res, void *cuda_stream);

/* Correct nfields independent fields in one run: every pass of the loop
 * covers all fields still violating a constraint (one launch per stage per
 * pass over all of them).  Arrays of per-field device pointers / values are
 * HOST arrays of length nfields; edits_out / edits_cap may be NULL.  Each
 * field's result equals what exactz_correct returns for it alone.
 * Returns the first error met (per-field status in res[i]). */
int exactz_correct_batch(uint32_t nfields, const float *const *f, const float *const *fhat,
                         const exactz_dims *d, const float *xi, const exactz_opts *opts,
                         float *const *g_out, exactz_edit *const *edits_out,
                         const uint64_t *edits_cap, exactz_result *res, void *cuda_stream);

/* ---- reusable workspace (allocation outside the timed / serving path) ---- */

typedef struct exactz_workspace exactz_workspace;

/* Plan device memory for up to nfields fields of the given dims (a HOST
 * array).  Any later call may pass fields whose vertex count does not exceed
 * the planned one field by field.  Returns NULL on failure (no device or out
 * of memory). */
exactz_workspace *exactz_workspace_create(uint32_t nfields, const exactz_dims *dims);
void exactz_workspace_destroy(exactz_workspace *ws);
/* Device bytes held by the workspace. */
uint64_t exactz_workspace_bytes(const exactz_workspace *ws);

/* exactz_correct_batch on a workspace (same arguments and results).  With
 * host_buffers = 1 every f / fhat / g_out / edits_out pointer is a HOST
 * pointer: the call copies inputs in and results out (both inside the call,
 * on cuda_stream), using device staging buffers held by the workspace. */
int exactz_ws_correct(exactz_workspace *ws, uint32_t nfields, const float *const *f,
                      const float *const *fhat, const exactz_dims *d, const float *xi,
                      const exactz_opts *opts, float *const *g_out,
                      exactz_edit *const *edits_out, const uint64_t *edits_cap,
                      exactz_result *res, void *cuda_stream, int host_buffers);

/* Correct a sequence of nitems host-resident fields of one shape d, one after
 * another on the workspace, each as exactz_correct would alone (Alg. 1 to
 * its fixpoint; opts for all, xi[i] per field), with the copies of the
 * neighbouring fields overlapping each correction: while field i runs on
 * cuda_stream, field i+1's f and f_hat are copied in on a copy-in stream and
 * field i-1's g and edit records copied out on a copy-out stream (two device
 * slots of inputs and outputs, held by the workspace, grown on first use).
 *   f[i], fhat[i]  HOST arrays of d.nx*d.ny*d.nz floats (pinned for overlap; read)
 *   g_out[i]       HOST array of as many floats (written)
 *   edits_out[i]   HOST array of edits_cap[i] records, or NULL (edits_out and
 *                  edits_cap may be NULL: no edit lists)
 *   res[i]         per-field result (zeroed for fields not reached)
 * The copy-in stream starts after the work queued on cuda_stream before the
 * call; the call returns with every copy landed.  Output arrays may be shared
 * between fields (the copies out run in field order: the last one stays).
 * Errors: EXACTZ_EINVAL (a null pointer, xi[i] <= 0 or not finite, bad dims
 * or opts) before any copy; otherwise the first error of a field stops the
 * sequence there (earlier fields' results are complete) and is returned;
 * EXACTZ_ECAP as for exactz_correct (the sequence goes on). */
int exactz_ws_correct_sequence(exactz_workspace *ws, uint32_t nitems, const float *const *f,
                               const float *const *fhat, exactz_dims d, const float *xi,
                               const exactz_opts *opts, float *const *g_out,
                               exactz_edit *const *edits_out, const uint64_t *edits_cap,
                               exactz_result *res, void *cuda_stream);

/* The same for a sequence of nsteps batches of nfields fields each (the
 * paper has no counterpart): step s corrects fields s*nfields .. s*nfields +
 * nfields - 1 together, as exactz_ws_correct would, field j having dims[j]
 * in every step.  Step s+1's inputs are copied in and step s-1's outputs
 * copied out while step s is corrected (two device slots of the whole batch,
 * held by the workspace and grown on first use: 24 bytes per vertex plus the
 * edit records).  f, fhat, xi, g_out, edits_out, edits_cap and res hold
 * nsteps*nfields entries, step-major, with the meanings above; field j's
 * edit records get a region of the largest edits_cap[s*nfields + j] over
 * the steps.  Errors as above, per step (EXACTZ_EINVAL also for nfields = 0).
 * exactz_ws_correct_sequence is the case nfields = 1. */
int exactz_ws_correct_batch_sequence(exactz_workspace *ws, uint32_t nsteps, uint32_t nfields,
                                     const exactz_dims *dims, const float *const *f,
                                     const float *const *fhat, const float *xi, const exactz_opts *opts,
                                     float *const *g_out, exactz_edit *const *edits_out,
                                     const uint64_t *edits_cap, exactz_result *res, void *cuda_stream);

/* Statistics of the last exactz_ws_correct on a workspace.  stage_ms holds
 * CUDA-event times on the call's stream when opts.profile was 1 (else 0):
 * [0] set-up stencil kernel, [1] critical-point compaction, [2] radix sort
 * (with EXACTZ_EVENTS_ORIGINAL also the extremum-graph set-up), [3] first
 * pass (pair check, apply, bookkeeping), [4] the loop, [5] residual and
 * status, [6] the edit list's time beyond [5] (it runs beside the residual
 * check) and the reflection of increasing edits, [7] whole call on the device. */
typedef struct {
    uint64_t kernel_launches; /* kernels the call executed (graph bodies counted per pass) */
    uint64_t passes;          /* edit passes run for the slowest field, including the last check */
    uint64_t total_critical;  /* listed critical points over all fields (saddles only with EXACTZ_EVENTS_ORIGINAL) */
    uint64_t sum_requests;    /* deduplicated edit requests over all passes */
    uint64_t sum_tiles;       /* tiles re-checked by frontier passes (0 for PLAIN) */
    uint64_t sum_pairs;       /* CP pairs re-checked by frontier passes (0 for PLAIN) */
    float stage_ms[8];
    /* PLAIN and FRONTIER with opts.profile = 1: summed CUDA-event times of the
     * loop passes' kernels (after the first pass), [0] vertex checks (rules R1,
     * R2), [1] CP-pair checks (R3), [2] edits; loop_passes = passes timed. */
    float loop_kernel_ms[3];
    uint32_t reserved;
    uint64_t loop_passes;
    uint64_t sum_visits;      /* vertices checked by frontier passes (the dirty vertices of their tiles) */
} exactz_stats;

int exactz_ws_stats(const exactz_workspace *ws, exactz_stats *out);

/* ---- launch-schedule autotuning (the paper has no counterpart) ---- */

/* The per-pass kernels' launch schedule on a workspace: resident blocks per SM
 * of the tile-check, tile-apply and CP-pair kernels, and whether each block
 * takes a contiguous chunk of the tile list (1) or every grid-th tile (0).
 * Defaults: 48, 32, 8, 0 (what the search picks on the 512^3 and 1024^3
 * workloads and on the 256-field batch).  The schedule never changes any result. */
typedef struct {
    uint32_t stencil_blocks_per_sm;
    uint32_t apply_blocks_per_sm;
    uint32_t pairs_blocks_per_sm;
    uint32_t chunked_schedule;
    float best_ms; /* exactz_ws_autotune: time of the best schedule (ms) */
} exactz_tuning;

int exactz_ws_get_tuning(const exactz_workspace *ws, exactz_tuning *out);
/* Values out of range (blocks per SM outside 1..64, chunked_schedule > 1)
 * return EXACTZ_EINVAL. */
int exactz_ws_set_tuning(exactz_workspace *ws, const exactz_tuning *t);

/* Pick the schedule for these fields by timing whole corrections on
 * cuda_stream (coordinate descent over the four knobs, best of `repeats`
 * runs, 0 = 2).  The fields are device arrays as for exactz_ws_correct; the
 * call allocates scratch outputs for the trial runs and frees them.  The
 * chosen schedule stays with the workspace and is written to *out. */
int exactz_ws_autotune(exactz_workspace *ws, uint32_t nfields, const float *const *f,
                       const float *const *fhat, const exactz_dims *d, const float *xi,
                       const exactz_opts *opts, void *cuda_stream, uint32_t repeats,
                       exactz_tuning *out);

/* ---- inspection of the set-up stage (Sec. 3.2, Sec. 4.3) ---- */

/* Per-vertex descriptor of field h (device arrays of n entries):
 *   bits 0-3  rank (0..14) of the steepest-ascent vertex of the closed
 *             neighbourhood, bits 4-7 that of the steepest-descent vertex,
 *             where ranks list the closed neighbourhood in increasing vertex
 *             index (7 = the vertex itself);
 *   bits 8-21 lower-link mask (bit s for neighbour rank s < 7, s+1 otherwise);
 *   bit 22    saddle; bit 23 critical point.
 * type_out (may be NULL): 0 regular, 1 minimum, 2 maximum, 4|8 join|split saddle. */
int exactz_classify(const float *h, exactz_dims d, uint32_t *desc_out, uint8_t *type_out,
                    void *cuda_stream);

/* Critical points of f sorted by (value, index) into order_out (device array
 * of at least n uint64); *count_out (HOST) receives their number. */
int exactz_cp_order(const float *f, exactz_dims d, uint64_t *order_out, uint64_t *count_out,
                    void *cuda_stream);

/* ---- edit stream: the stored form of a result (Sec. 3.3; storage accounting) ---- */

/* The edits of a result as they are stored next to the base compressor's
 * output: one edit-count byte per vertex (0..N decrements of Delta, N+1 = the
 * lossless bound fl(f - xi)) and the lossless values in index order.  From
 * f_hat, xi and N these reproduce g bit for bit (exactz_decode_edits).
 *
 * Encode: edits (DEVICE, n_edits records in strictly ascending idx, as the
 * correction writes them); kcodes_out (DEVICE, n bytes); lossless_out (DEVICE,
 * room for lossless_cap floats); *n_lossless_out (HOST) = their number.
 * Returns EXACTZ_EINVAL for a malformed list (not ascending, idx >= n, k
 * outside 1..N+1, lossless flag not equal to k == N+1; kcodes_out is then
 * unspecified) and EXACTZ_ECAP when the lossless values exceed lossless_cap
 * (none written).  Allocates a few bytes of device scratch per 4096 items. */
int exactz_encode_edits(const exactz_edit *edits, uint64_t n_edits, uint64_t n, uint32_t N, uint8_t *kcodes_out,
                        float *lossless_out, uint64_t lossless_cap, uint64_t *n_lossless_out, void *cuda_stream);

/* Decode: g_out (DEVICE, n floats) = f_hat (DEVICE) after k_i steps of
 * fl(g - Delta) (fl(g + Delta) for direction = EXACTZ_EDITS_INCREASING),
 * Delta = fl(xi / N), or, where k_i = N+1, the next lossless value (DEVICE, in
 * index order).  Returns EXACTZ_EINVAL for a code above N+1, for xi <= 0, N
 * outside 1..254 or an unknown direction. */
int exactz_decode_edits(const float *fhat, uint64_t n, float xi, uint32_t N, uint32_t direction,
                        const uint8_t *kcodes, const float *lossless, float *g_out, void *cuda_stream);

/* ---- allocation-free variant for small fields (the paper has no counterpart) ---- */

/* Largest field (in vertices) and the fixed device scratch behind
 * exactz_correct_noalloc. */
#define EXACTZ_NOALLOC_MAX_VERTICES (1u << 18)
#define EXACTZ_NOALLOC_SCRATCH_BYTES (32ull << 20)

/* exactz_correct for fields of at most EXACTZ_NOALLOC_MAX_VERTICES vertices
 * (for example 64^3) that allocates no memory: no cudaMalloc, cudaFree,
 * pinned host memory, graph or event objects.  It is meant for callers that
 * cannot allocate device memory in the middle of their work: applications
 * that reserve the whole device memory up front for their own pool
 * (simulations, in-situ analysis), where a cudaMalloc would fail or take
 * memory promised elsewhere, and loops that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree.  The caller still passes the inputs
 * and outputs (device pointers, as for exactz_correct).
 *
 * The passes are driven from the host: every pass reads a few bytes of loop
 * state back and synchronises cuda_stream, and the call returns only after
 * its work on the stream has finished.
 *
 * Scratch: one EXACTZ_NOALLOC_SCRATCH_BYTES array of static device storage
 * inside this library, held by every GPU that loads the library until the
 * process exits (the largest accepted field uses about 19 MiB of it: about
 * 72 bytes per vertex).  The first call on a device looks up that array's
 * device address (a set-up step).  All calls share the array and it keeps the
 * previous call's contents; each call clears what must start at zero.  Calls
 * whose GPU work overlapped would race on the array: within one process they
 * are serialised by a lock, which each call releases only after its stream
 * has drained (on error returns too).
 * A GRAPH or FUSED mode request runs the same passes as FRONTIER (identical results);
 * opts->profile is ignored.  EXACTZ_EVENTS_ORIGINAL needs set-up storage sized
 * by the field's extremum graph and is refused (EXACTZ_EINVAL); increasing
 * edits are offered (their reflected fields live in the same scratch).
 * Returns EXACTZ_ESIZE for larger fields, otherwise as exactz_correct. */
int exactz_correct_noalloc(const float *f, const float *fhat, exactz_dims d, float xi,
                           const exactz_opts *opts, float *g_out, exactz_edit *edits_out,
                           uint64_t edits_cap, exactz_result *res, void *cuda_stream);

/* ---- request server with continuous batching (the paper has no counterpart) ---- */

/* A server corrects fields submitted one at a time from HOST memory.  It owns
 * one device arena planned from budget_bytes (about 1/8 for edit records, the
 * rest at 60 bytes per resident vertex) and a host thread that runs the passes
 * of Algorithm 1 over every resident field at once.  At each pass boundary it
 * admits queued requests in submission order while a field slot and arena room
 * are free (a request that does not fit waits; later ones wait behind it),
 * and retires fields whose loop ended: their residual check, status and edit
 * list are computed, g and the edit list are copied into the caller's host
 * buffers, and the room is freed.  Every field runs the passes of
 * EXACTZ_MODE_FRONTIER; its result is bit-identical to exactz_correct's for
 * the same input and options, whatever else is resident. */
typedef struct exactz_server exactz_server;

typedef struct {
    uint64_t budget_bytes; /* device memory for the arena (>= 64 MiB) */
    uint32_t max_fields;   /* resident fields at most (1..4096) */
    uint32_t reserved;
    exactz_opts opts;      /* N, max_iters, want_edit_list and direction (decreasing or increasing
                              edits) for every request (N = 0: defaults); mode ignored; events must be 0 */
} exactz_server_config;

typedef struct {
    uint64_t submitted, completed;
    uint64_t passes;            /* passes the server ran */
    uint64_t resident, queued;  /* now */
    uint64_t max_resident;      /* most fields in one pass */
    uint64_t admitted_vertices; /* sum of admitted fields' vertices */
    uint64_t capacity_vertices; /* largest admissible field, in vertices */
    uint64_t device_bytes;      /* device memory held */
    uint64_t kernel_launches;   /* kernels launched so far */
    double busy_s;              /* host time spent in passes */
    int32_t error;              /* 0, or the CUDA failure that stopped the server (EXACTZ_ENODEV) */
    int32_t reserved;
    uint64_t cancelled;         /* requests withdrawn by exactz_server_cancel */
} exactz_server_info;

/* Returns NULL without a device, on a bad configuration or when the arena
 * cannot be allocated.  The server uses the calling thread's current device. */
exactz_server *exactz_server_create(const exactz_server_config *cfg);

/* Queue one field.  f, fhat: HOST arrays of n floats; g_out: HOST array of n
 * floats; edits_out: HOST array of edits_cap records, or NULL.  The buffers
 * must stay valid and untouched until the request's result is taken (poll or
 * wait returned 1); page-locked buffers copy fastest.  *ticket identifies the
 * request.  Returns EXACTZ_EINVAL (bad dims, xi, pointers, or the server has
 * stopped), EXACTZ_ESIZE (larger than an empty arena holds) or EXACTZ_OK.
 * Invalid values (NaN, out of bound) are reported in the result's status. */
int exactz_server_submit(exactz_server *s, const float *f, const float *fhat, exactz_dims d, float xi,
                         float *g_out, exactz_edit *edits_out, uint64_t edits_cap, uint64_t *ticket);

/* 1: done -- *res (status < 0 for invalid input; n_edits > edits_cap means
 * the list was truncated) and *latency_s (submission to results in host
 * memory) are filled and the ticket is released.  0: not yet (wait: timed
 * out; timeout_s < 0 waits without limit).  EXACTZ_EINVAL: unknown ticket;
 * EXACTZ_ENODEV: the server stopped on a CUDA failure. */
int exactz_server_poll(exactz_server *s, uint64_t ticket, exactz_result *res, double *latency_s);
int exactz_server_wait(exactz_server *s, uint64_t ticket, double timeout_s, exactz_result *res,
                       double *latency_s);
int exactz_server_stats(exactz_server *s, exactz_server_info *out);
/* Withdraws a request that is still queued (not yet admitted): returns 1, and
 * the server never reads its inputs or writes its outputs again (the caller
 * may free them); the ticket is then unknown to poll / wait.  Returns 0 when
 * the request was already admitted or finished (its result comes as usual)
 * and EXACTZ_EINVAL for an unknown ticket. */
int exactz_server_cancel(exactz_server *s, uint64_t ticket);
/* Finishes every submitted request, then frees the server.  Results not yet
 * taken are discarded (their host buffers hold them). */
void exactz_server_destroy(exactz_server *s);

/* Library build / device information (host string, static storage). */
const char *exactz_version(void);

/* ---- testing aid: allocation-failure injection (the paper has no counterpart) ---- */

/* After `skip` more successful device allocations inside this library, the
 * next `count` fail as if cudaMalloc had run out of memory (no cudaMalloc is
 * called for them); count = 0 disarms it.  Process-wide; for tests that check
 * that every call reports EXACTZ_ENOMEM (workspace and server creation return
 * NULL), frees what it had allocated, and that the library works afterwards.
 * Always returns EXACTZ_OK. */
int exactz_debug_fail_allocations(uint64_t skip, uint64_t count);

#ifdef __cplusplus
}
#endif
#endif /* EXACTZ_H */
