/*
 * gbaes -- bulk AES on NVIDIA GB300 (sm_103a): the C ABI.
 *
 * What it computes: the AES block cipher (FIPS-197; 128-bit blocks, 128/192/256-bit
 * keys, 10/12/14 rounds) on many independent 16-byte blocks, as described in
 * Section 2.1 of "AES Encryption and Decryption Using Direct3D 10 API" (Chiuta),
 * with each round in the fused T-table form of Eq. 1 (SubBytes, ShiftRows and
 * MixColumns folded into four 32-bit table lookups XORed with the round key),
 * plus the parallel modes of Section 3 (ECB, CTR, CBC decryption).
 *
 * Conventions shared by every call:
 *  - A block is 16 bytes read "exactly as found in memory" (Section 3): four
 *    little-endian 32-bit words, byte 4c+r of the block is row r of column c.
 *  - Data pointers named in/out are DEVICE pointers (cudaMalloc, torch CUDA
 *    tensors, managed memory, or page-locked host memory from cudaHostAlloc /
 *    cudaHostRegister).  The caller owns them.  Each must be 16-byte aligned
 *    (AES_ERR_ALIGN) and [ptr, ptr + 16*nblocks) must lie inside one such
 *    allocation (AES_ERR_ARG otherwise; unregistered pageable host memory is
 *    refused because its extent cannot be checked).  The library checks this
 *    on the host before launching, so a bad pointer is an error code, not a
 *    GPU fault.
 *  - in == out (in place) is allowed unless a call says otherwise; any other
 *    overlap of the two ranges is rejected (AES_ERR_ARG).
 *  - nblocks == 0 returns AES_OK and launches nothing.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that launch work are asynchronous on that stream and
 *    return AES_OK once the work is queued; completion is observed through the
 *    stream.  No call here synchronises the device unless it says so.
 *  - Keys and IVs are HOST pointers, read during the call only.
 *  - There is no padding (Section 2.1 leaves the padding values unspecified);
 *    lengths are whole blocks.  There is no CPU fallback: without a usable
 *    CUDA device, launching calls return AES_ERR_CUDA.
 *  - On failure a call returns a negative AES_ERR_* code and records a message
 *    that aes_last_error() returns (per thread).
 */
#ifndef GBAES_H_
#define GBAES_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AES_OK 0
#define AES_ERR_ARG (-1)     /* bad pointer, size, flag or overlapping ranges */
#define AES_ERR_KEYSIZE (-2) /* bits not in {128, 192, 256} */
#define AES_ERR_ALIGN (-3)   /* a data pointer is not 16-byte aligned */
#define AES_ERR_CUDA (-4)    /* a CUDA runtime call or kernel launch failed */
#define AES_ERR_BUDGET (-5)  /* request larger than a server's memory budget */
#define AES_ERR_NOMEM (-6)   /* host or device allocation failed */
#define AES_ERR_DEVICE (-7)  /* a kernel reported an error through its status word */
#define AES_ERR_STATE (-8)   /* object used in the wrong state (e.g. closed server) */

/* Kernel variants for aes_ecb_ex / aes_set_kernel. */
#define AES_KERNEL_TABLE 0     /* Eq. 1 T-table kernel, tables in shared memory: the replicated
                                  tables, or the compact ones for calls too small to fill the GPU */
#define AES_KERNEL_BITSLICED 1 /* Boolean-circuit S-box over bit planes of 32 blocks */
#define AES_KERNEL_TABLE_COMPACT 2    /* T-table kernel with each table stored once (4-5 KiB of shared
                                         memory, cheap to fill; lookups may meet bank conflicts), any
                                         size; its launch shape is its own (threads and
                                         blocks_per_thread are ignored) */
#define AES_KERNEL_TABLE_REPLICATED 3 /* T-table kernel with 32 lane copies of each table (bank-conflict
                                         free, 128-160 KiB to fill per CTA), any size */

/* Counter layouts for aes_ctr_xcrypt (Section 3, CTR mode). */
#define AES_CTR_BE128 0     /* IV is one big-endian 128-bit integer (NIST SP 800-38A) */
#define AES_CTR_LE32_CARRY 1 /* IV is four little-endian 32-bit words x,y,z,w; the
                                block index is added to x with a carry into y, z, w
                                (the counter of Section 3's CTR listing) */

/* Opaque key context: the host copy of the expanded encryption schedule and of
 * the equivalent-inverse decryption schedule.  Immutable after creation, so one
 * context may be used from several threads and streams at once. */
typedef struct aes_ctx aes_ctx;

/* Key expansion (round keys K_i of Eq. 1; FIPS-197 KeyExpansion, which Section
 * 2.1 defers to).  key: HOST pointer to bits/8 bytes; bits in {128,192,256}.
 * Computes the (Nr+1) x 4-word encryption schedule and the decryption schedule
 * of the equivalent inverse cipher (same round keys in reverse order, with
 * InvMixColumns applied to rounds 1..Nr-1).  Needs no GPU.  Returns NULL on
 * error (see aes_last_error()).  Free with aes_free_ctx. */
aes_ctx* aes_expand_key(const uint8_t* key, int bits);

/* Frees a context.  The caller must ensure no queued work still uses it (the
 * launching calls copy the schedule into the launch, so a context may be freed
 * as soon as the launching call has returned).  NULL is ignored. */
void aes_free_ctx(aes_ctx* ctx);

/* Key size in bits of a context (128/192/256), or AES_ERR_ARG. */
int aes_ctx_bits(const aes_ctx* ctx);

/* ECB encryption of nblocks independent blocks (Section 3: one block per
 * pixel; Eq. 1 for rounds 1..Nr-1, an S-box-only last round).  in/out:
 * device pointers, 16*nblocks bytes each; in == out allowed. */
int aes_encrypt_ecb(const aes_ctx* ctx, const void* in, void* out, size_t nblocks, void* stream);

/* ECB decryption (Section 2.1: the inverse cipher), run as the equivalent
 * inverse cipher with inverse T-tables; same arguments as aes_encrypt_ecb. */
int aes_decrypt_ecb(const aes_ctx* ctx, const void* in, void* out, size_t nblocks, void* stream);

/* ECB with an explicit kernel choice, for benchmarking and tuning.
 * decrypt: 0/1.  kernel: AES_KERNEL_*.  threads: CTA size, a multiple of 32 in
 * [64, 1024] (0 = default; checked, but the bitsliced kernel always runs
 * 128-thread CTAs, its shape fixed by its register budget).
 * blocks_per_thread: 1, 2 or 4 for the table kernel (0 = default; the
 * bitsliced kernel always holds 32 blocks per pair of lanes). */
int aes_ecb_ex(const aes_ctx* ctx, int decrypt, const void* in, void* out, size_t nblocks, int kernel,
               int threads, int blocks_per_thread, void* stream);

/* CTR mode (Section 3): out_i = in_i XOR E_K(counter(first_block + i)) for
 * i < nblocks.  iv: HOST pointer to 16 bytes.  counter_kind: AES_CTR_*.  The
 * counter arithmetic is modulo 2^128; block indices are 64-bit, so
 * first_block + nblocks - 1 must not exceed 2^64 - 1 (AES_ERR_ARG).  Encryption
 * and decryption are the same call.  in == out allowed. */
int aes_ctr_xcrypt(const aes_ctx* ctx, const uint8_t* iv, int counter_kind, uint64_t first_block, const void* in,
                   void* out, size_t nblocks, void* stream);

/* CBC decryption (Section 3, Eq. 2; the first block is chained to the IV on
 * the GPU rather than on the CPU): out_i = D_K(in_i) XOR in_{i-1}, in_{-1} =
 * iv (HOST pointer to 16 bytes).  To decrypt a long message in pieces, pass
 * the last ciphertext block of the previous piece as iv.  in and out must not
 * overlap at all (each output depends on two input blocks). */
int aes_cbc_decrypt(const aes_ctx* ctx, const uint8_t* iv, const void* in, void* out, size_t nblocks, void* stream);

/* ---------------------------------------------------------------- batched
 * Many messages, each with its own key, key size and direction, in ONE
 * persistent launch (pattern: batching).  The paper issues one draw per
 * buffer and notes that per-operation overhead dominates small inputs
 * (Section 3.1; Section 4 advises against small messages); batching amortises
 * that overhead over thousands of messages.  Messages may be in-place
 * (in_base+in_off == out_base+out_off); otherwise outputs must not overlap
 * any other message's input or output (not checked). */
typedef struct aes_msg_desc {
    uint64_t in_off;    /* byte offset of the message's input from in_base (multiple of 16) */
    uint64_t out_off;   /* byte offset of its output from out_base (multiple of 16) */
    uint64_t nblocks;   /* 16-byte blocks (0 = nothing to do) */
    uint32_t key_index; /* index into the ctxs array */
    uint32_t decrypt;   /* 0 = encrypt, 1 = decrypt */
} aes_msg_desc;

typedef struct aes_batch_plan aes_batch_plan;

/* Builds a reusable plan: validates every descriptor (AES_ERR_ARG /
 * AES_ERR_ALIGN), groups messages by direction and key size, tiles the
 * flattened blocks (one tile = 128 * blocks_per_thread blocks, taken by one
 * warp; CTAs of `threads` threads; blocks_per_thread 1, 2, 4 or 8, with 8
 * needing threads <= 512; 0, 0 = 1024, 2) and uploads the tile table, message table and every context's two
 * schedules to one device allocation on the current device (cudaMalloc,
 * synchronous).  msgs and ctxs are HOST arrays, read during the call only.
 * Returns NULL on error. */
aes_batch_plan* aes_batch_plan_create(const aes_msg_desc* msgs, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx,
                                      int threads, int blocks_per_thread);

/* Launches a plan on `stream`: resets the plan's tile counters, then one
 * persistent kernel (one CTA per SM; its warps take tiles independently).  in_base/out_base: device buffers of
 * in_bytes/out_bytes bytes that must cover every message (AES_ERR_ARG).  Two
 * launches of the same plan must not run concurrently (they share its tile
 * counter); stream-ordered repeats are fine. */
int aes_batch_plan_launch(aes_batch_plan* plan, const void* in_base, size_t in_bytes, void* out_base,
                          size_t out_bytes, void* stream);

/* Same as aes_batch_plan_launch through a CUDA graph captured on first use
 * (counter reset + kernel) and replayed afterwards; new base pointers update
 * the captured kernel's arguments.  Same concurrency rule. */
int aes_batch_plan_launch_graph(aes_batch_plan* plan, const void* in_base, size_t in_bytes, void* out_base,
                                size_t out_bytes, void* stream);

/* Plan statistics (any output may be NULL). */
int aes_batch_plan_info(const aes_batch_plan* plan, uint64_t* total_blocks, uint32_t* ntiles, uint32_t* tile_blocks);

/* Frees a plan (synchronises with the device through cudaFree). */
void aes_batch_plan_free(aes_batch_plan* plan);

/* One-shot batch: plan tables in stream-ordered scratch (cudaMallocAsync /
 * cudaFreeAsync on `stream`), one launch with 1024 threads x 2 blocks per
 * tile.  Same arguments and rules as the plan calls.  The tables are uploaded
 * from a host copy that is freed when the call returns, so a stream that is
 * being captured into a CUDA graph is refused (AES_ERR_STATE); for graphs use
 * a plan and aes_batch_plan_launch_graph. */
int aes_ecb_batch(const aes_msg_desc* msgs, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx, const void* in_base,
                  size_t in_bytes, void* out_base, size_t out_bytes, void* stream);

/* Batch without device allocation (the paper has no counterpart; this entry
 * point exists for callers that cannot call cudaMalloc -- code whose device
 * memory belongs to another runtime or allocator, or latency-critical paths
 * that must not pay for an allocation).  Same arguments, rules and kernel as
 * aes_ecb_batch, but the plan tables and the tile counter live in one fixed
 * 8 MiB device array inside this library instead of freshly allocated memory:
 *  - Nothing is allocated on the device: no cudaMalloc/cudaFree, no memory
 *    pool.  The array exists on every GPU that loads the library, until exit.
 *  - A batch whose tables exceed 8 MiB (512 bytes per key context, 32 bytes per
 *    message, 4 bytes per 2048-block tile, plus 256) is rejected with
 *    AES_ERR_ARG; the 10,000-message, 10,000-key batch needs about 5.6 MiB.
 *  - The first call in each CUDA context (normally once per device, in its
 *    primary context) looks up the array's device address there
 *    (cudaGetSymbolAddress) and keeps it for that context.
 *  - Every call shares the one array and overwrites it (the tile counter is
 *    re-zeroed by each call's upload).  Calls whose work overlaps on the GPU
 *    -- on different streams, or from different host threads -- race on it;
 *    issue them on one stream or otherwise order them. */
int aes_ecb_batch_noalloc(const aes_msg_desc* msgs, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx,
                          const void* in_base, size_t in_bytes, void* out_base, size_t out_bytes, void* stream);

/* ------------------------------------------------------- host pipeline
 * ECB on data in host memory (Section 3 copies every texture over the bus and
 * Fig. 3 shows those copies dominating small inputs).  A pipeline picks how the
 * data reaches the SMs:
 *  - AES_PIPE_STAGED: `depth` device staging slots of chunk_bytes each (0, 0 =
 *    64 MiB x 4), each with its own stream; chunks go round-robin over the
 *    slots (copy in, in-place table kernel, copy out), so copies in both
 *    directions overlap the kernels.
 *  - AES_PIPE_DIRECT: no staging; one table-kernel launch reads the host input
 *    and writes the host output over the host link (on a coherent link such as
 *    NVLink-C2C the faster of the two).  chunk_bytes and depth are checked but
 *    not used. */
#define AES_PIPE_STAGED 0
#define AES_PIPE_DIRECT 1
typedef struct aes_pipeline aes_pipeline;

/* Creates a pipeline on the current device; staged mode allocates its slots
 * (cudaMalloc) and streams.  chunk_bytes: multiple of 16; depth: 1..16; mode:
 * AES_PIPE_STAGED or AES_PIPE_DIRECT.  NULL on error (AES_ERR_ARG for a bad
 * argument, before any CUDA call). */
aes_pipeline* aes_pipeline_create_ex(size_t chunk_bytes, int depth, int mode);

/* aes_pipeline_create_ex(chunk_bytes, depth, AES_PIPE_STAGED). */
aes_pipeline* aes_pipeline_create(size_t chunk_bytes, int depth);

/* ECB over nblocks blocks from host_in to host_out: page-locked host memory
 * (cudaHostAlloc / cudaHostRegister; device memory also works), each covering
 * 16*nblocks bytes (AES_ERR_ARG otherwise); host_in == host_out allowed.
 * Asynchronous on `stream`: the stream waits for every chunk's copy-out (staged)
 * or for the kernel (direct), so host_out is complete once the stream is.  One
 * staged pipeline serves one call at a time (calls from several threads
 * serialise on it); a direct pipeline holds no state between calls. */
int aes_pipeline_ecb(aes_pipeline* pipe, const aes_ctx* ctx, int decrypt, const void* host_in, void* host_out,
                     size_t nblocks, void* stream);

/* Waits for the pipeline's streams, then frees it.  NULL is ignored. */
void aes_pipeline_free(aes_pipeline* pipe);

/* ---------------------------------------------------------------- serving
 * Continuous-batching server (pattern: serving).  Section 3.1 finds per-call
 * overhead dominating small inputs and Section 4 advises against small
 * messages on the GPU; the server batches requests as they arrive instead:
 * a scheduler thread admits requests in arrival order while the input+output
 * bytes of admitted, unfinished requests fit the device-memory budget, packs
 * them into one batched-kernel launch per free stream slot (batches on
 * different slots overlap on the device), and completes a batch's requests as
 * soon as its event fires, freeing budget and slot for requests that arrived
 * meanwhile.  Key schedules stay resident on the device for the server's
 * life.  Request data are device pointers owned by the caller, which must keep
 * them valid until the request completes.  AES_SERVER_RESIDENT (below)
 * replaces the per-batch launches with one kernel that stays on the GPU. */

#define AES_SERVER_DRYRUN 1 /* no GPU work: a batch completes dryrun_batch_us after its launch */

/* Resident mode: instead of one batched-kernel launch per micro-batch, one
 * kernel stays on the GPU (one CTA per SM) and takes requests as they are
 * admitted.  The scheduler cuts each request into tiles of at most threads *
 * blocks_per_thread blocks (spread over the idle CTAs, at least 256 blocks
 * each), writes them into a ring in mapped page-locked memory and publishes
 * them with a release store; in each CTA a producer warp takes tiles with
 * tickets from an atomic counter and stages the next tile's record while the
 * compute threads encipher the current one, and a completer warp counts
 * finished tiles and appends each finished request to a completion queue in
 * page-locked memory, which the scheduler reads.  No
 * launch, copy or event per request.  The scheduler stops the kernel after
 * resident_idle_us without work and before resident_lifetime_ms (its bound on
 * the GPU) have passed, and relaunches it when work arrives.  While it runs it
 * holds every SM, so other kernels on the device wait for it, and so does a
 * device-wide synchronisation (cudaDeviceSynchronize).  Request inputs must be
 * complete in device memory when submitted.  With AES_SERVER_DRYRUN, a host
 * thread runs the kernel's protocol instead (each tile takes dryrun_batch_us).
 * Stats: `batches` counts kernel launches, batch_msgs is 1. */
#define AES_SERVER_RESIDENT 2

/* Pins the scheduler thread to the last CPU of the process's affinity set and
 * the replay thread to the one before it (pthread_setaffinity_np), so that
 * neither migrates; other threads of the process may still share those CPUs. */
#define AES_SERVER_PIN_THREADS 4

typedef struct aes_server aes_server;

typedef struct aes_server_config {
    uint64_t budget_bytes;      /* in+out bytes in flight (0 = 8 GiB) */
    int32_t nstreams;           /* stream slots, 1..64 (0 = 4) */
    int32_t flags;              /* AES_SERVER_* */
    int32_t threads;            /* batched-kernel CTA size, or the resident kernel's compute threads per CTA
                                   (at most 512; two control warps come on top) (0 = 512) */
    int32_t blocks_per_thread;  /* 1, 2 or 4 (0 = 1; resident mode: 2) */
    uint32_t max_batch_msgs;    /* requests per batch (0 = 4096) */
    uint32_t dryrun_batch_us;   /* AES_SERVER_DRYRUN only: simulated time a batch spends "on the GPU" */
    uint64_t max_batch_blocks;  /* blocks per batch, also the largest request (0 = 2^22) */
    uint32_t resident_idle_us;     /* AES_SERVER_RESIDENT: the kernel is stopped after this long without work (0 = 2000) */
    uint32_t resident_lifetime_ms; /* ... and restarted before this long after its launch (0 = 10000) */
    uint32_t ring_tiles;           /* tile records per direction, a power of two (0 = 65536); must hold the
                                      largest request */
    uint32_t ring_items;           /* requests in flight per direction, a power of two (0 = 16384) */
    uint32_t resident_restart_pct; /* the scheduler restarts the kernel at this % of its lifetime (0 = 80;
                                      1..1000; above 100 the kernel's own bound ends it first, and the
                                      scheduler recovers the tiles it left) */
} aes_server_config;

typedef struct aes_server_request {
    uint64_t id;        /* caller's tag, returned in the completion */
    const void* in;     /* device pointer, 16-byte aligned, 16*nblocks bytes */
    void* out;          /* device pointer; in == out allowed */
    uint64_t nblocks;
    uint32_t key_index; /* index into the server's keys */
    uint32_t decrypt;   /* 0 = encrypt, 1 = decrypt */
    double arrival_s;   /* replay only: scheduled arrival, seconds after the replay starts */
} aes_server_request;

typedef struct aes_server_completion {
    uint64_t id;
    int32_t status;      /* AES_OK, or the error the request failed with */
    uint32_t batch_msgs; /* requests in its batch (1 in resident mode) */
    double arrival_s;    /* arrival (scheduled, for replays) on the server clock, seconds */
    double launch_s;     /* launch of its batch */
    double done_s;       /* when its completion was observed */
} aes_server_completion;

typedef struct aes_server_stats {
    uint64_t submitted, completed, failed, rejected, batches;
    uint64_t max_inflight_bytes; /* peak admitted in+out bytes (never above the budget) */
    uint64_t max_queue;          /* peak requests waiting for admission */
    uint64_t max_batch_msgs;
    uint64_t budget_bytes;
    uint64_t recovered_tiles;    /* resident mode: tiles re-published after the kernel's own bound ended it */
    uint64_t lost_completions;   /* completions dropped because no host memory was left to hold them
                                    (aes_server_poll never returns these; 0 unless memory ran out) */
} aes_server_stats;

/* Host-thread diagnostics of a server, for latency tails.  Times in ns; the
 * "_at_ns" fields say when the worst case happened, in ns on the server's clock
 * (which starts at creation).  The scheduler reads its own CPU time,
 * context-switch and page-fault counts (getrusage) every 16 passes and after
 * any pass that comes more than 50 us after the one before; between two
 * readings lies a window.  A window far longer than the CPU time in it, with
 * involuntary switches, is time the thread was descheduled; with voluntary
 * ones, time it blocked (a lock, a CUDA call, a page fault) or yielded. */
typedef struct aes_server_diag {
    uint64_t sched_passes;              /* scheduler passes */
    uint64_t sched_worst_window_ns;     /* longest window in which the scheduler had work waiting throughout */
    uint64_t sched_worst_window_cpu_ns; /* CPU time the scheduler got in that window */
    uint64_t sched_worst_window_invol;  /* involuntary context switches (preemptions) in that window */
    uint64_t sched_worst_window_vol;    /* voluntary context switches (blocking waits, yields) in that window */
    uint64_t sched_worst_window_at_ns;  /* when that window began */
    uint64_t sched_worst_window_minflt; /* page faults in that window: minor (no I/O), */
    uint64_t sched_worst_window_majflt; /* and major */
    uint64_t sched_invol;               /* involuntary context switches of the scheduler over the server's life */
    uint64_t lock_wait_max_ns[3];       /* the scheduler's longest wait for the submission, completion and stats locks */
    uint64_t lock_wait_at_ns[3];
    uint64_t cuda_call_max_ns;          /* the scheduler's longest CUDA call (event or stream query, launch) */
    uint64_t cuda_call_at_ns;
    uint64_t stream_queries[2];         /* resident mode: stream queries made to confirm an end every CTA had
                                           marked, and because the kernel showed no sign of life for 50 ms */
    uint64_t sched_phase_max_ns[5];     /* the scheduler's longest pass phase: taking submissions, completions,
                                           kernel or event queries, admission, launches and statistics (in
                                           launch-per-batch mode, completions count under the queries and
                                           admission under launches) */
    uint64_t sched_phase_at_ns[5];
    uint64_t inbox_hold_max_ns[2];      /* longest hold of the submission lock: by the scheduler, by a submitter */
    uint64_t producer_late_max_ns;      /* replay: latest hand-over after the first due request's arrival time */
    uint64_t producer_late_at_ns;
    uint64_t producer_late_invol;       /* replay: involuntary switches since the thread's reading before that */
    uint64_t producer_invol;            /* replay: involuntary context switches over all replays */
    uint64_t producer_check_max_ns;     /* replay: longest host check of one request (driver pointer queries),
                                           made when aes_server_replay is called */
    uint64_t producer_check_at_ns;
    int64_t sched_cpu;                  /* CPU the scheduler thread is pinned to (AES_SERVER_PIN_THREADS), else -1 */
    int64_t producer_cpu;               /* CPU the replay thread is pinned to, else -1 */
    uint64_t sched_minflt;              /* minor page faults of the scheduler thread (sampled with its windows) */
    uint64_t producer_minflt;           /* replay: minor page faults over all replays */
} aes_server_diag;

/* Copies the server's host-thread diagnostics. */
int aes_server_get_diag(aes_server* server, aes_server_diag* out);

/* Creates a server on the current device with nkeys resident key contexts
 * (copied; the caller may free them afterwards) and starts its scheduler
 * thread.  config may be NULL for the defaults.  NULL on error.
 * The server keeps the data its threads touch on every pass (its own state,
 * queues, key copies, replay arrays, completions and the top of each thread's
 * stack) in page-locked host memory, which the kernel's memory compaction
 * cannot move: ~7 MiB to start, plus ~100 bytes per request of each replay,
 * held until aes_server_destroy. */
aes_server* aes_server_create(const aes_ctx* const* keys, size_t nkeys, const aes_server_config* config);

/* Queues one request (arrival = now).  Checks its pointers and sizes on the
 * host; a request whose in+out bytes exceed the budget, or whose blocks
 * exceed max_batch_blocks, is refused with AES_ERR_BUDGET. */
int aes_server_submit(aes_server* server, const aes_server_request* req);

/* Starts a producer thread that submits reqs[i] at arrival_s[i] seconds after
 * the call (open loop: late submissions keep their scheduled arrival time, so
 * queueing delay is counted).  The array is copied and every request is
 * checked during this call (the caller must keep its buffers valid until the
 * requests complete); a request that fails its check completes with its error
 * at its arrival time.  The call also makes room for all n completions
 * (40 bytes each, page-locked host memory, kept by the server until it is
 * destroyed), so the server's threads do not allocate while the replay runs.
 * One replay at a time. */
int aes_server_replay(aes_server* server, const aes_server_request* reqs, size_t n);

/* Waits for the replay thread (stop_early != 0: ends it after its current request). */
int aes_server_replay_join(aes_server* server, int stop_early);

/* Waits until every submitted request has completed (timeout_s < 0: forever).
 * AES_ERR_STATE on timeout. */
int aes_server_drain(aes_server* server, double timeout_s);

/* Moves up to max completions (at most 2^31-1 per call) into out, oldest first;
 * returns how many. */
int aes_server_poll(aes_server* server, aes_server_completion* out, size_t max);

/* Copies the server's counters. */
int aes_server_get_stats(aes_server* server, aes_server_stats* out);

/* Cancels request `id` if it is still waiting for admission: it completes at
 * once with AES_ERR_STATE.  A request already admitted to a batch runs to
 * completion (its GPU work cannot be withdrawn).  Unknown ids are ignored. */
int aes_server_cancel(aes_server* server, uint64_t id);

/* Test hook: the batch with this index (0-based, in launch order) fails as if
 * its launch had returned an error; its requests complete with
 * AES_ERR_DEVICE and the server carries on. */
int aes_server_inject_fault(aes_server* server, uint64_t batch_index);

/* Stops the replay, finishes every queued request, stops the scheduler and
 * frees the server.  NULL is ignored. */
void aes_server_destroy(aes_server* server);

/* ---------------------------------------------------------------- routing
 * Several servers behind one submission point: independent replicas (one
 * server per GPU, each created with its device current) sharing nothing on
 * the data path.  The router only chooses a server per request and merges
 * their completions; it neither owns nor destroys the servers.  A resident
 * server holds every SM of its GPU, so put one resident server per GPU. */

#define AES_ROUTE_LEAST_LOADED 0 /* the server with the fewest unfinished requests (ties: round robin); every
                                    server must be able to read the request's buffers */
#define AES_ROUTE_BY_DEVICE 1    /* the least loaded of the servers on the device that holds the request's
                                    input (input not in device memory, or no server there: of all) */

typedef struct aes_router aes_router;

/* servers: n >= 1 distinct servers (copied array).  NULL on error. */
aes_router* aes_router_create(aes_server* const* servers, size_t n, int policy);

/* Routes one request (aes_server_submit on the chosen server).  Returns the
 * index of the chosen server (>= 0) or that server's error. */
int aes_router_submit(aes_router* router, const aes_server_request* req);

/* Moves up to max completions of every server into out; returns how many. */
int aes_router_poll(aes_router* router, aes_server_completion* out, size_t max);

/* aes_server_drain on every server with the same timeout. */
int aes_router_drain(aes_router* router, double timeout_s);

/* Frees the router (not the servers).  NULL is ignored. */
void aes_router_destroy(aes_router* router);

/* Default kernel variant for aes_encrypt_ecb / aes_decrypt_ecb (process-wide;
 * AES_KERNEL_TABLE at start).  Returns the previous variant or AES_ERR_ARG. */
int aes_set_kernel(int which);

/* Default launch shape of the table kernel for one (key size, direction):
 * threads per CTA (multiple of 32, 64..1024) and blocks per thread (1/2/4).
 * The autotuner calls this with the shape it measured fastest. */
int aes_set_tuning(int bits, int decrypt, int threads, int blocks_per_thread);

/* Reads (and with clear != 0 resets) the library's device status word on the
 * current device: 0 when no kernel has reported an error.  Synchronises the
 * device.  Returns the status (>= 0) or AES_ERR_CUDA. */
int aes_device_status(int clear);

/* Message for the last failed call on this thread ("" if none). */
const char* aes_last_error(void);

/* ---------------------------------------------------------------- host only
 * These run on the CPU alone (no GPU needed) and expose the library's own
 * tables and schedules so their host logic can be tested without a device. */

/* Writes the expanded schedules as little-endian words: enc_rk and dec_rk each
 * receive 4*(Nr+1) uint32 (either may be NULL).  Returns Nr or a negative code. */
int aes_key_schedule(const uint8_t* key, int bits, uint32_t* enc_rk, uint32_t* dec_rk);

/* Copies the library's generated tables: Te0 and Td0 of Eq. 1 (256 words each;
 * T_k = rotl(T_0, 8k)), the S-box and the inverse S-box (256 bytes each).  Any
 * pointer may be NULL.  Returns AES_OK. */
int aes_host_tables(uint32_t* te0, uint32_t* td0, uint8_t* sbox, uint8_t* inv_sbox);

/* Host-only view of a batch's tiling: validates the descriptors like
 * aes_batch_plan_create and writes, for each tile of tile_blocks blocks, the
 * caller's index of the first message that tile touches (tiles in plan order:
 * encryption groups 128/192/256, then decryption groups).  first_msg may be
 * NULL; otherwise it holds cap entries.  Returns the number of tiles or a
 * negative code.  Needs no GPU. */
int aes_batch_tiles(const aes_msg_desc* msgs, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx, int tile_blocks,
                    uint32_t* first_msg, size_t cap);

#ifdef __cplusplus
}
#endif

#endif /* GBAES_H_ */
