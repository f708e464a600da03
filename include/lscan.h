/*
 * lscan.h -- C ABI of the GB300 single-pass scan library (liblscan.so).
 *
 * Operation (LightScan, Section 1): given an associative operator (+) and
 * x_0..x_{N-1}, the inclusive scan writes y_j = x_0 (+) ... (+) x_j and the
 * exclusive scan writes y_j = x_0 (+) ... (+) x_{j-1}, with y_0 = identity
 * (0 for add, INT32_MIN / -infinity for max).
 *
 * Method (Section 4): the array is cut into tiles of L elements; each tile is
 * scanned in registers by one thread block (thread-serial scan, warp-shuffle
 * Hillis-Steele scan of thread totals as in Algorithm 2, block scan of warp
 * totals as in Algorithm 3), the carry between tiles travels through per-tile
 * status words in L2 (Section 4.3, Algorithm 4; here either the paper's
 * chained neighbour-to-neighbour hand-off or a decoupled look-back), and each
 * tile applies its carry and stores y once (Section 4.4, Algorithm 5).  Every
 * element of x is read once and every element of y written once (Section 1,
 * contribution (i)); y may equal x (in-place, Section 4.5).
 *
 * Conventions shared by every entry point:
 *  - x, y are DEVICE pointers owned by the caller; any element-aligned address
 *    is accepted (16-byte-aligned x and y take the TMA bulk-copy path).
 *  - y == x is allowed when input and output elements have the same size;
 *    any other overlap of [x, x+n) and [y, y+n) returns LSCAN_ERR_INVALID.
 *  - n == 0 returns LSCAN_OK without a launch; n < 0 is LSCAN_ERR_INVALID.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous: argument errors are returned at once; errors the
 *    device detects (a carry or tile-ring wait that ran out of time) are
 *    latched in the stream's device error word and returned by
 *    lscan_stream_status().
 *  - Scratch (per-tile status words, tile ticket, epoch and error word) is
 *    owned by the library, one set per (device, stream), grown on demand with
 *    cudaMalloc and released by lscan_shutdown().  Growing it is not allowed
 *    while the stream is being captured; call lscan_reserve() first.
 *  - Different streams may be used from different host threads concurrently;
 *    two calls on the same stream are ordered by the stream.  A host thread
 *    with no current CUDA context gets the current device's primary context
 *    bound by its first call (as any CUDA runtime call would bind it).
 *  - The scan, single-CTA and digit-offset kernels are launched with
 *    programmatic stream serialization: their thread blocks may be
 *    scheduled while the previous kernel of the stream is finishing, but
 *    each waits for that kernel to complete (and its writes to be visible)
 *    before it reads or writes global memory, so stream order holds.
 *  - Output dtype equals the input dtype, except bf16 add, which writes fp32
 *    unless lscan_options.out_dtype asks for bf16.
 *  - int32 add wraps modulo 2^32; max keeps the earlier element on ties
 *    (so +0/-0 ties keep the first one's bits); NaN inputs are outside the
 *    contract.
 */
#ifndef LSCAN_H
#define LSCAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { LSCAN_ADD = 0, LSCAN_MAX = 1 } lscan_op;

/* LSCAN_I64 and LSCAN_F64 are the paper's other two types (Section 5,
 * Table 2): int64 add wraps mod 2^64; double add runs in double in the tile
 * and in the carry chain (precision DEFAULT or F64_CARRY only). */
typedef enum {
    LSCAN_I32 = 0,
    LSCAN_F32 = 1,
    LSCAN_BF16 = 2,
    LSCAN_I64 = 3,
    LSCAN_F64 = 4
} lscan_dtype;

typedef enum {
    LSCAN_OK = 0,
    LSCAN_ERR_INVALID = 1,     /* bad argument (pointer, size, overlap, ...) */
    LSCAN_ERR_UNSUPPORTED = 2, /* combination not built (op, dtype, config) */
    LSCAN_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    LSCAN_ERR_TIMEOUT = 4,     /* a device-side carry wait ran out of time */
    LSCAN_ERR_NOMEM = 5,       /* device allocation or HBM budget exhausted */
    LSCAN_ERR_BUSY = 6,        /* scratch growth needed during stream capture */
    LSCAN_ERR_DEVICE = 7       /* the device latched an unclassified error */
} lscan_status;

/* Float-add precision of the cross-tile carry chain (the one step whose
 * rounding error grows with N / L).  Integer and max scans are exact and
 * ignore this field.  Bounds against the exact prefix, with
 * S_j = sum of |x_i| over the scanned prefix: |err_j| <= 1e-5 S_j for the
 * F32 (measured, not guaranteed: its worst case grows with the number of
 * carry hops), F64 and DF paths; <= 2.5e-7 S_j for COMPENSATED. */
typedef enum {
    LSCAN_PREC_DEFAULT = 0,     /* = LSCAN_PREC_DF_CARRY */
    LSCAN_PREC_F32_CARRY = 1,   /* fp32 in tile, fp32 carry chain (plain) */
    LSCAN_PREC_F64_CARRY = 2,   /* fp32 in tile, FP64 carry chain */
    LSCAN_PREC_COMPENSATED = 3, /* compensated in tile (an exact two-sum per
                                   element into an fp32 hi/lo pair),
                                   double-float carry */
    LSCAN_PREC_DF_CARRY = 4     /* fp32 in tile, double-float carry chain: a
                                   normalised fp32 hi/lo pair (48-bit
                                   significand) added with two-sum
                                   arithmetic; no FP64 instruction on the
                                   carry path */
} lscan_precision;

/* Inter-tile carry protocol (Section 4.3). */
typedef enum {
    LSCAN_CARRY_AUTO = 0,     /* the measured best (= LSCAN_CARRY_LOOKBACK) */
    LSCAN_CARRY_LOOKBACK = 1, /* a tile combines its predecessors' published */
                              /* aggregates until it meets an inclusive prefix */
    LSCAN_CARRY_CHAINED = 2   /* a tile waits for its left neighbour's */
                              /* inclusive prefix and passes on its own (Alg. 4) */
} lscan_carry;

/* Optional per-call settings; pass NULL for all defaults.  Zero in any field
 * means "default / tuned". */
typedef struct lscan_options {
    int32_t out_dtype;   /* 0 or -1 = default; LSCAN_F32 / LSCAN_BF16 select
                            the output of a bf16 add */
    int32_t precision;   /* lscan_precision */
    int32_t carry;       /* lscan_carry */
    int32_t config;      /* 0 = tuned; 1..lscan_num_configs() pick a
                            bulk-copy tile configuration */
    int32_t max_ctas;    /* cap on persistent CTAs, 0 = occupancy x SMs */
    int32_t carry_in_type; /* 0: carry_in is one output element; 1: it holds
                              a value of the kind's carry type
                              (lscan_carry_bytes bytes, aligned to that size),
                              as lscan_reduce and lscan_carry_combine make */
    /* Single-array scans only (not in the paper: the carry-in of a scan
     * sharded over devices, where shard g starts from the total of the shards
     * before it).  NULL = the operator's identity.  Otherwise a device
     * pointer to ONE element of the output type (carry_in_type 0) or to one
     * value of the kind's carry type (carry_in_type 1), read by the kernel in
     * stream order: inclusive y_j = c (+) x_0 (+) ... (+) x_j, exclusive
     * y_0 = c and y_j = c (+) x_0 (+) ... (+) x_{j-1}.  It must be aligned
     * to its size; batched calls with a carry-in return
     * LSCAN_ERR_INVALID. */
    const void *carry_in;
} lscan_options;

/* Single-array scan (Section 4; Algorithm 1).  x: n input elements, y: n
 * output elements (layout: contiguous, element type from dtype/out_dtype).
 * With the tile configuration left to the library (config 0), arrays of at
 * most 4096 elements run a single-CTA kernel that has no inter-tile carry
 * and uses no scratch (not in the paper: a latency path for tiny arrays). */
lscan_status lscan_inclusive(lscan_op op, lscan_dtype dtype, const void *x,
                             void *y, int64_t n, void *stream);
lscan_status lscan_exclusive(lscan_op op, lscan_dtype dtype, const void *x,
                             void *y, int64_t n, void *stream);
/* Same with options and an inclusive flag (1 = inclusive, 0 = exclusive). */
lscan_status lscan_scan(lscan_op op, lscan_dtype dtype, int inclusive,
                        const void *x, void *y, int64_t n,
                        const lscan_options *opts, void *stream);

/* Single-array scan of an array in HOST memory (not in the paper, whose
 * arrays are on the device).  hx: n input elements in host memory; hy: n
 * output elements in host memory (element types as for lscan_scan); hy == hx
 * is allowed when the two element sizes are equal, partial overlap returns
 * LSCAN_ERR_INVALID.  Page-locked memory (cudaHostAlloc / cudaHostRegister)
 * gets full copy bandwidth and overlap; pageable memory is accepted, but its
 * copies are staged by the CUDA driver and overlap less.
 *  - The array moves in chunks of `chunk` elements through three device
 *    slots: chunk k is copied in while chunk k-1 is scanned on `stream` and
 *    chunk k-2 is copied out, on two internal streams.  chunk = 0 lets the
 *    library choose: chunks that double from 2^20 to 2^23 elements at the
 *    start and halve again over the last 2^24, so that the first copy-in
 *    and the last copy-out, which overlap nothing, are short.  Chunk
 *    k > 0 starts from the inclusive total of chunks 0..k-1, handed on in
 *    the kind's carry type (FP64 for the float adds with an FP64 carry), so
 *    the results meet the same rules and bounds as lscan_scan over the whole
 *    array.
 *  - opts as for lscan_scan; opts->carry_in (a DEVICE pointer to one output
 *    element) is the carry-in of chunk 0.
 *  - Asynchronous on stream: the copies start after the work already queued
 *    on stream, and work queued on stream afterwards runs after the last
 *    element of hy is written.  hx and hy must stay valid until then.
 *  - The device slots, 3 x chunk (at most 2^23 for chunk = 0) x (input +
 *    output element size) bytes, are owned by the library per (device,
 *    stream), grow on demand (after the previous call's copies finish) and
 *    are freed by lscan_shutdown.
 *  - Not capturable: returns LSCAN_ERR_UNSUPPORTED while stream is being
 *    captured.  Device-side carry timeouts latch on stream as for
 *    lscan_scan (lscan_stream_status).  After LSCAN_ERR_CUDA or
 *    LSCAN_ERR_NOMEM the contents of hy are unspecified. */
lscan_status lscan_scan_host(lscan_op op, lscan_dtype dtype, int inclusive,
                             const void *hx, void *hy, int64_t n,
                             const lscan_options *opts, int64_t chunk,
                             void *stream);

/* The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory when they scan: a memory-pool or
 * allocator implementation that is itself servicing an allocation, code under
 * a framework that forbids allocations outside its own pool, or a latency-
 * critical path where cudaMalloc (which may synchronise or fail) is not
 * acceptable.  It runs the same single-array scan as lscan_scan with default
 * options, but its scratch (control block + per-tile status words) is a
 * fixed array compiled into the library: 2 MiB + 512 B that every GPU which
 * loads the library keeps until the process exits.
 *  - n is limited by that array: at most 262144 status words.  Launches use
 *    tile configuration 2 whatever the tuning table says (16 KiB input
 *    tiles; 2 status words per tile for every kind of lscan_scan), so the
 *    limit is 2^29 elements for int32 and fp32 (4096-element tiles), 2^30 for
 *    bf16 input (8192-element tiles) and 2^28 for int64 and double
 *    (2048-element tiles); with x or y not 16-byte aligned the plain-load
 *    configuration's tiles are half as long and so is the limit (2^28 int32).
 *    Larger n returns LSCAN_ERR_INVALID without launching.  Arrays of at most
 *    4096 elements take the single-CTA kernel and use no scratch.
 *  - The first call on a device is a set-up call: it looks up the array (under
 *    CUDA's lazy module loading, the moment the driver loads the module and
 *    places the array) and clears it with cudaMemsetAsync on `stream`.  Make
 *    that first call at initialisation, outside any context that must not
 *    allocate.
 *  - Every call shares the array (it keeps the last call's contents; each
 *    launch re-arms it for the next one).  Calls that overlap on the GPU race
 *    on it: keep them on one stream or synchronise between them.
 *  - It allocates nothing (no cudaMalloc, cudaFree or allocating library
 *    call).  Every device-side wait is bounded, so a call cannot hang; a wait
 *    that ran out latches the array's error word, which
 *    lscan_noalloc_status() reports. */
lscan_status lscan_scan_noalloc(lscan_op op, lscan_dtype dtype, int inclusive,
                                const void *x, void *y, int64_t n,
                                void *stream);
/* Waits for `stream`, then returns and clears the error word of the current
 * device's fixed array used by lscan_scan_noalloc: LSCAN_OK,
 * LSCAN_ERR_TIMEOUT (a device wait of some no-allocation launch ran out:
 * its output is wrong) or LSCAN_ERR_CUDA.  Reads by symbol, allocating
 * nothing.  (The paper has no counterpart.) */
lscan_status lscan_noalloc_status(void *stream);

/* ------------------------------------------------------- sharded scans
 * A scan of one array split into contiguous shards over several devices
 * (not in the paper, whose arrays live on one GPU: its inter-block carry of
 * Section 4.3 lifted one level up).  Reduce-then-scan, 3N bytes:
 *   1. each device: lscan_reduce(shard) -> its total, in the carry type;
 *   2. the caller's collective all-gathers the P totals (lscan_carry_bytes
 *      bytes each);
 *   3. each device: lscan_carry_combine(totals of the shards before it) ->
 *      its offset (on the host), copied to the device and passed to
 *      lscan_scan as carry_in with carry_in_type = 1.
 * The carry type keeps the precision path's accuracy across the boundary:
 * uint32/uint64 wrapping sums, int32/int64/float maxima (double max as an
 * order-preserving int64 key), fp32 for the fp32 carry, FP64 for the FP64
 * carry and double add, a normalised fp32 (hi, lo) pair for the
 * double-float and compensated paths. */

/* Size in bytes (4 or 8) of the carry type of the scan lscan_scan would run
 * for (op, dtype, opts: out_dtype and precision); 0 if unsupported. */
int32_t lscan_carry_bytes(lscan_op op, lscan_dtype dtype,
                          const lscan_options *opts);
/* d_total (DEVICE, lscan_carry_bytes bytes, aligned to that size, not
 * overlapping x) = x_0 (+) ... (+) x_{n-1} in the kind's carry type (the
 * identity for n = 0).  One pass over x (16-byte loads when x is 16-byte
 * aligned; any element-aligned x is accepted).  Per 16-byte chunk the
 * elements are folded in the scan's in-tile arithmetic and the chunks in the
 * carry arithmetic; float max keeps the first occurrence (+0 / -0).  The
 * CTAs' partials are combined through the scan's inter-block carry chain
 * (status slots of the stream's scratch, shared with lscan_scan; a bounded
 * wait that runs out is reported by lscan_stream_status as
 * LSCAN_ERR_TIMEOUT).  Asynchronous on stream. */
lscan_status lscan_reduce(lscan_op op, lscan_dtype dtype, const void *x,
                          int64_t n, const lscan_options *opts, void *d_total,
                          void *stream);
/* HOST: h_out = totals[0] (+) ... (+) totals[count - 1] in the kind's carry
 * arithmetic, earlier operands first (the identity for count = 0).
 * h_totals: count values of lscan_carry_bytes bytes each, in host memory.
 * Needs no GPU. */
lscan_status lscan_carry_combine(lscan_op op, lscan_dtype dtype,
                                 const lscan_options *opts,
                                 const void *h_totals, int32_t count,
                                 void *h_out);

/* Batched scan of n_seg independent arrays stored back to back in x (and y):
 * segment s is elements [offsets[s], offsets[s+1]).  d_offsets is a DEVICE
 * array of n_seg+1 int64, non-decreasing, offsets[0] = 0 and
 * offsets[n_seg] = n_total (n_total passed by the caller so that no
 * device-to-host read is needed).  One persistent launch; tiles span segment
 * boundaries and the carry restarts at every segment head.  Malformed
 * offsets never cause an out-of-bounds access; they give undefined results.
 * (Not in the paper: the batched pattern of this library.) */
lscan_status lscan_batched(lscan_op op, lscan_dtype dtype, int inclusive,
                           const void *x, void *y, const int64_t *d_offsets,
                           int64_t n_seg, int64_t n_total,
                           const lscan_options *opts, void *stream);

/* A scan captured once into a CUDA graph (one kernel node) with a private
 * scratch set, replayed by lscan_graph_launch.  The pointers, sizes and
 * options are fixed at creation.  Replays of one graph must be ordered (same
 * stream or synchronised) because they share that scratch.  The kernel
 * re-arms the scratch at the end of each launch, so a replay needs no memset.
 * (CUDA-graph capture is this library's batched pattern, not the paper's.) */
typedef struct lscan_graph lscan_graph;
lscan_status lscan_graph_create_scan(lscan_op op, lscan_dtype dtype,
                                     int inclusive, const void *x, void *y,
                                     int64_t n, const lscan_options *opts,
                                     lscan_graph **out);
lscan_status lscan_graph_create_batched(lscan_op op, lscan_dtype dtype,
                                        int inclusive, const void *x, void *y,
                                        const int64_t *d_offsets, int64_t n_seg,
                                        int64_t n_total,
                                        const lscan_options *opts,
                                        lscan_graph **out);
lscan_status lscan_graph_launch(lscan_graph *g, void *stream);
/* Synchronises the device and returns/clears the graph's device error. */
lscan_status lscan_graph_status(lscan_graph *g);
void lscan_graph_destroy(lscan_graph *g);

/* ---------------------------------------------------------------- serving
 * A continuous-batching scan service on the current device (not in the
 * paper; the serving pattern of this library).  The server owns ONE device
 * allocation of hbm_budget_bytes: per-stream scratch plus a pool for request
 * outputs and client buffers, so nothing is allocated while serving.
 * Requests wait in a FIFO admission queue (one per size-class lane, see
 * lscan_server_set_lanes) until the pool can hold their output; a scheduler
 * thread per stream keeps its two launch slots busy (the second queued behind
 * the first, so the device does not wait for the host between launches),
 * each running one persistent launch over the admitted requests of one
 * (op, dtype, inclusive) kind and lane -- up to 8192 tiles for the bulk
 * lane by default -- so kinds overlap on the device and later arrivals join
 * the next launch.  n_streams bulk streams plus one small-lane stream, each
 * with its own scheduler thread.
 * While batches are in flight the scheduler thread polls their completion
 * events (it sleeps when the server is idle).  Times are microseconds on the
 * host's steady clock since server creation; launch and completion times
 * come from CUDA events. */
typedef struct lscan_server lscan_server;
typedef struct lscan_req_stats {
    double submit_us;  /* submit() call (replay: scheduled arrival) */
    double admit_us;   /* output allocated from the pool */
    double launch_us;  /* its batch started on the device */
    double done_us;    /* its batch finished on the device */
    void *y;           /* output (server-allocated ones: until release) */
    int64_t n;
    int32_t status;          /* lscan_status of the request */
    int32_t batch_requests;  /* requests in the same launch */
} lscan_req_stats;
typedef struct lscan_trace_req {
    int32_t op, dtype, inclusive, reserved;
    const void *x;      /* device input */
    int64_t n;
    double arrival_us;  /* offset from the start of the replay */
} lscan_trace_req;

/* NULL on failure (bad arguments, budget below the scratch reserve + 1 MiB,
 * or the allocation failed). */
lscan_server *lscan_server_create(size_t hbm_budget_bytes, int n_streams);
/* Finishes in-flight batches, fails never-admitted requests, frees all. */
void lscan_server_destroy(lscan_server *srv);
/* hold != 0: keep admitting and queueing requests but start no new launch
 * (batches already launched finish); hold == 0: launch what has queued,
 * batched by kind.  Lets a client gather a burst into few launches.
 * Destroying a held server still runs everything it admitted. */
lscan_status lscan_server_hold(lscan_server *srv, int hold);
/* Size-class lanes.  Requests of at most small_max_elems elements (default
 * 2^14) of the kinds the resident kernel scans (int32 add and max, fp32 and
 * bf16 max, fp32 and bf16 add with the default double-float carry and fp32
 * output, int64 add and max, double add and max) take the resident lane: a
 * persistent kernel on reserve_sms SMs (default 4, 0 .. 64; 0 reserves none
 * and the kernel shares the SMs) takes each request from a ring of
 * descriptors in host memory mapped for the device, scans it with one CTA
 * and writes its done word -- no launch per request; the submitting thread
 * publishes the request itself.  The kernel leaves after 20 ms without work
 * and is launched again when work arrives.  Other requests form bulk
 * batches of at most bulk_batch_tiles tiles (default 32768, 1 .. 65536),
 * launched for (SMs - reserve_sms) SMs.  small_max_elems = 0 puts every
 * request in the bulk lane.  Applies to requests submitted afterwards.
 * (Not in the paper.) */
lscan_status lscan_server_set_lanes(lscan_server *srv, int64_t small_max_elems,
                                   int64_t bulk_batch_tiles, int32_t reserve_sms);
/* Client buffers from the pool (count against the budget); NOMEM if full. */
lscan_status lscan_server_alloc(lscan_server *srv, size_t bytes, void **dptr);
lscan_status lscan_server_free(lscan_server *srv, void *dptr);
/* x: device input (any element-aligned address; 16-byte aligned inputs and
 * outputs take the bulk-copy path).  y: device output, or NULL to have the
 * server allocate it from the pool at admission (reported in the stats and
 * kept until lscan_server_release).  Returns at once with a ticket.  One
 * request holds at most 512 MiB of input (65536 tiles of 8 KiB); larger n
 * returns LSCAN_ERR_INVALID. */
lscan_status lscan_server_submit(lscan_server *srv, lscan_op op,
                                 lscan_dtype dtype, int inclusive,
                                 const void *x, void *y, int64_t n,
                                 uint64_t *ticket);
/* Blocks until the request finished; returns its status. */
lscan_status lscan_server_wait(lscan_server *srv, uint64_t ticket,
                               lscan_req_stats *out);
/* Non-blocking: LSCAN_ERR_BUSY while the request is still pending. */
lscan_status lscan_server_poll(lscan_server *srv, uint64_t ticket,
                               lscan_req_stats *out);
/* Forgets a finished request and frees a server-allocated output. */
lscan_status lscan_server_release(lscan_server *srv, uint64_t ticket);
/* Open-loop load replay: a native thread submits trace[i] at its arrival
 * time (outputs allocated by the server), completions are collected and
 * released in completion order; out[i] receives each request's stats and
 * *wall_us the time from the first arrival to the last completion.  One
 * replay at a time per server: a second concurrent call returns
 * LSCAN_ERR_BUSY. */
lscan_status lscan_server_replay(lscan_server *srv,
                                 const lscan_trace_req *trace, int64_t n_req,
                                 lscan_req_stats *out, double *wall_us);

/* Waits for the stream, then returns and clears its latched device error:
 * LSCAN_OK or LSCAN_ERR_TIMEOUT (LSCAN_ERR_CUDA if a CUDA call failed). */
lscan_status lscan_stream_status(void *stream);

/* Makes sure the stream's scratch holds status words for scans of up to
 * max_elems elements (all configurations), so that later calls on the
 * stream never allocate (e.g. before CUDA-graph capture). */
lscan_status lscan_reserve(void *stream, int64_t max_elems);

/* Frees every scratch buffer, captured graph and tuning entry. */
void lscan_shutdown(void);

const char *lscan_strerror(lscan_status s);
const char *lscan_version(void);

/* Number of kernels this library has launched in this process (used to
 * count launches inside a timed region). */
uint64_t lscan_launch_count(void);

/* Upper bound, in nanoseconds, on any device-side wait (carry flags, bulk
 * copy barriers).  A wait that runs out sets the stream's error word to
 * LSCAN_ERR_TIMEOUT and the kernel finishes without hanging.  Default 1 s;
 * limits below 20 us act as 20 us (waits check the limit only after that). */
lscan_status lscan_set_wait_limit_ns(uint64_t ns);

/* Fault injection for tests: the next launch on any stream skips publishing
 * the status word of tile `tile` (-1 disables), so that its successors'
 * waits run out and the timeout path is exercised on the host's request. */
lscan_status lscan_debug_skip_publish(int64_t tile);

/* Autotuner (not in the paper, whose K and T are fixed per dtype, Section
 * 5.1).  Times every bulk-copy tile configuration built for the mode --
 * items per thread x consumer warps x ring stages x tiles per ticket x
 * status-slot width, lscan_num_configs() of them for single arrays, the
 * first six for batched scans -- on the caller's buffers (a single-array
 * scan, or a batched one when d_offsets is given): two untimed launches,
 * then `reps` launches each timed with CUDA events on `stream`, the median
 * kept.  The paper's chained carry (Algorithm 4) is then timed at the
 * fastest configuration when the array has at most 4096 tiles (beyond that
 * its one L2 round trip per tile in series cannot compete).  The fastest
 * (configuration, carry) is recorded for this (op, dtype, precision/output
 * kind, mode, log2(n) class) and used by later calls that leave config and
 * carry at 0.  y is overwritten with the scan of x.  LSCAN_ERR_UNSUPPORTED
 * if the buffers are not 16-byte aligned (only the plain-load
 * configuration applies).  out (may be NULL) receives the measurements. */
#define LSCAN_TUNE_MAX_CONFIGS 32
typedef struct lscan_tune_result {
    int32_t config;          /* fastest configuration (1-based) */
    int32_t carry;           /* its lscan_carry (LOOKBACK or CHAINED) */
    float ms;                /* its median launch time, ms */
    int32_t default_config;  /* the built-in default for this kind and mode */
    float default_ms;        /* the default's median time, ms */
    int32_t n_timed;         /* configurations timed */
    float chained_ms;        /* chained carry at `config`, 0 if not timed */
    float ms_by_config[LSCAN_TUNE_MAX_CONFIGS]; /* look-back, per config
                                 (index config - 1); 0 = not built */
} lscan_tune_result;
lscan_status lscan_autotune(lscan_op op, lscan_dtype dtype, int inclusive,
                            const void *x, void *y, int64_t n,
                            const int64_t *d_offsets, int64_t n_seg,
                            const lscan_options *opts, int reps, void *stream,
                            lscan_tune_result *out);
/* The tuning table as JSON ({"lscan_tune": 1, "entries": [[kind, mode,
 * size_class, config, carry], ...]}, only entries that differ from the
 * defaults; four-field entries load with carry 0 = auto);
 * it is also loaded automatically from $LSCAN_TUNE_FILE on first use. */
lscan_status lscan_tune_save(const char *path);
lscan_status lscan_tune_load(const char *path);
/* Back to the built-in defaults: each kind's fastest configuration on a
 * 2^28-element array on GB300, with the look-back carry. */
lscan_status lscan_tune_reset(void);

/* Stream compaction (a consumer of the scan; not in the paper): y receives,
 * in order, every x[j] whose flags[j] is nonzero, and *d_count (device
 * int64, 8-byte aligned) the number kept.  One pass: the flags are scanned
 * as 0/1 counts with the single-pass carry chain (Section 4.3) and each kept
 * element is written once, at its index = the exclusive prefix sum of the
 * flags.  x, y: n elements of dtype (any type: the bits are moved); flags: n
 * bytes; y must not overlap x or flags.  n = 0 sets *d_count to 0.
 * Asynchronous on stream; device waits report through lscan_stream_status. */
lscan_status lscan_select_flagged(lscan_dtype dtype, const void *x,
                                  const uint8_t *flags, void *y, int64_t n,
                                  int64_t *d_count, void *stream);

/* Radix-sort digit offsets (a consumer of the scan; not in the paper, which
 * lists parallel sorting among the applications of scan in Section 1; radix
 * sort is the sort built on it).  keys: n
 * unsigned integers of key_bytes (4 or 8) bytes in device memory, aligned
 * to key_bytes (16-byte-aligned keys are read with 16-byte loads).  Digit p
 * (p = 0 .. P-1, P = ceil(8 * key_bytes / digit_bits), lowest digit first)
 * of a key is (key >> (p * digit_bits)) & (2^digit_bits - 1).  With
 * B = 2^digit_bits, one pass over the keys writes
 *     d_offsets[p * B + v] = number of keys whose digit p is below v,
 * the exclusive scan of the digit-p histogram: where bucket v starts in a
 * stable counting-sort pass on digit p.  d_offsets: P * B int64 in device
 * memory, 8-byte aligned, not overlapping the keys.  Signed or float keys
 * are mapped to order-preserving unsigned keys by the caller.
 *  - digit_bits 1..8; 0 <= n <= 2^32 - 1; n = 0 writes zeros.  Otherwise
 *    LSCAN_ERR_INVALID, before any device work.
 *  - Scratch (2048 64-bit counters and a done word per (device, stream)) is
 *    owned by the library, zeroed when allocated and left zeroed by each
 *    launch; freed by lscan_shutdown.  Allocating it during stream capture
 *    returns LSCAN_ERR_BUSY (call once outside capture first).
 *  - Asynchronous on stream; one kernel launch, no device-side waits. */
lscan_status lscan_radix_offsets(const void *keys, int32_t key_bytes, int64_t n,
                                 int32_t digit_bits, int64_t *d_offsets,
                                 void *stream);

/* Describes a tile configuration: writes items per thread, consumer threads
 * per CTA, pipeline stages and tile length L for dtype `dtype`. */
lscan_status lscan_config_info(int32_t config, lscan_dtype dtype,
                               int32_t *items, int32_t *threads,
                               int32_t *stages, int32_t *tile);
int32_t lscan_num_configs(void);

#ifdef __cplusplus
}
#endif
#endif /* LSCAN_H */
