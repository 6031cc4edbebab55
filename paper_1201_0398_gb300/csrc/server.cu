// Continuous-batching AES server (pattern: serving).
//
// The paper advises against using the GPU for small messages because each
// operation pays a large fixed overhead (Section 3.1; Section 4).  The server
// answers that with continuous batching:
//
//  * Requests (key index, direction, device in/out pointers, length) arrive at
//    any time through aes_server_submit, or from a replay thread that issues a
//    recorded open-loop arrival schedule at its scheduled times.
//  * One scheduler thread admits requests in arrival order while the bytes in
//    flight (input + output of every admitted, unfinished request) stay within
//    the device-memory budget, packs them into a micro-batch, and launches it
//    through the batched kernel (batch.cu) on a free stream slot.  Batches on
//    different slots run concurrently on the device; as soon as a slot's event
//    fires, its requests complete, their bytes leave the budget, and the slot
//    takes the next batch -- requests that arrived meanwhile are admitted then.
//  * Expanded key schedules are resident on the device for the server's life;
//    a batch carries only its message and tile tables (a few hundred bytes per
//    request), copied from pinned staging on the slot's stream.
//  * Latency is completion time minus arrival time (the scheduled arrival for
//    replays, so a slow server cannot hide queueing delay).
//
// Resident mode (AES_SERVER_RESIDENT) replaces the per-batch launches: one
// kernel (resident.cu) stays on the GPU, the scheduler publishes each admitted
// request as tiles into a ring in page-locked memory and reads completions
// from a completion queue there (protocol in resident.h), and it stops and
// relaunches the kernel around idle periods.
//
// A dry-run mode replaces every CUDA call with a completion after a simulated
// service time (in resident mode, a host thread that runs the kernel's
// protocol), so the scheduling logic (admission, budget, batching, the ring,
// cancellation, fault handling, drain) can be exercised without a GPU.
#include <cuda_runtime.h>
#include <pthread.h>
#include <sched.h>
#include <sys/resource.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "batch_plan.h"
#include "resident.h"

namespace gbaes {

constexpr uint32_t kServerMagic = 0x53525652u;  // "SRVR"

struct Pending {
    aes_server_request r;
    double arrival;  // seconds on the server clock
};

// `bytes` of host memory with every page touched: page-locked by CUDA through
// `device`'s context (device >= 0; heap memory if the driver refuses) or plain
// heap memory (device < 0).  *locked says which; nullptr when out of memory.
// The caller's current device is left as it was.
static void* alloc_host(size_t bytes, int device, bool* locked) {
    void* p = nullptr;
    *locked = false;
    if (device >= 0) {
        int prev = -1;
        const bool swap = cudaGetDevice(&prev) == cudaSuccess && prev != device;
        if (swap) cudaSetDevice(device);
        if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable) == cudaSuccess) {
            *locked = true;
        } else {
            cudaGetLastError();
            p = nullptr;
        }
        if (swap) cudaSetDevice(prev);
        if (p) return p;
    }
    if (posix_memalign(&p, 4096, bytes) != 0) return nullptr;
    memset(p, 0, bytes);
    return p;
}

static void free_host(void* p, bool locked) {
    if (locked)
        cudaFreeHost(p);
    else
        free(p);
}

// Page-locked memory for the data the server's threads touch on every pass.
// The kernel's memory compaction moves ordinary pages, and a thread that
// touches a page while it is being moved sleeps until the move ends (measured
// on a GB300 node: scheduler and replay thread both in migration_entry_wait for
// 43-97 ms, every request in flight waiting with them); pages page-locked by
// CUDA are never moved.  HotPool hands out blocks in power-of-two size classes
// (64 B .. 2 MiB) carved from 4 MiB page-locked chunks and keeps freed blocks
// for reuse, so after warm-up the containers below allocate nothing new;
// larger blocks get page-locked allocations of their own, also kept for reuse
// until the pool goes (nothing is unpinned while the server runs).  In a dry run (no
// GPU) it uses ordinary heap memory, touched when carved.
class HotPool {
  public:
    explicit HotPool(int device) : device_(device) {}  // device < 0: heap memory (dry run)
    HotPool(const HotPool&) = delete;
    HotPool& operator=(const HotPool&) = delete;
    ~HotPool() {
        for (const auto& c : chunks_) free_host(c.first, c.second);
        for (const Big& b : big_) free_host(b.p, b.locked);
    }

    // (New memory is made with the lock released: the driver call can take
    // milliseconds, and the other thread's allocations need not wait for it.)
    void* allocate(size_t bytes) {
        const int c = size_class(bytes);
        std::unique_lock<std::mutex> lk(mu_);
        if (c < 0) {  // the smallest kept block that fits, else a new one
            const size_t want = (bytes + 4095) & ~(size_t)4095;
            size_t pick = big_.size();
            for (size_t i = 0; i < big_.size(); ++i)
                if (!big_[i].used && big_[i].bytes >= want && (pick == big_.size() || big_[i].bytes < big_[pick].bytes))
                    pick = i;
            if (pick < big_.size()) {
                big_[pick].used = true;
                return big_[pick].p;
            }
            lk.unlock();
            bool locked = false;
            void* p = alloc_host(want, device_, &locked);
            lk.lock();
            if (p) big_.push_back(Big{p, want, locked, true});
            return p;
        }
        const size_t sz = (size_t)64 << c;
        for (;;) {
            if (free_[c]) {
                void* p = free_[c];
                free_[c] = *static_cast<void**>(p);
                return p;
            }
            if (left_ >= sz) {
                void* p = cur_;
                cur_ += sz;
                left_ -= sz;
                return p;
            }
            lk.unlock();
            bool locked = false;
            void* chunk = alloc_host(kChunkBytes, device_, &locked);
            lk.lock();
            if (!chunk) return nullptr;
            chunks_.emplace_back(chunk, locked);
            if (left_ < sz) {  // (another thread may have made one meanwhile: the rest of this one stays unused)
                cur_ = static_cast<uint8_t*>(chunk);
                left_ = kChunkBytes;
            }
        }
    }

    void deallocate(void* p, size_t bytes) noexcept {
        if (!p) return;
        const int c = size_class(bytes);
        std::lock_guard<std::mutex> lk(mu_);
        if (c < 0) {  // kept for reuse: freeing page-locked memory can wait for the device
            for (Big& b : big_)
                if (b.p == p) b.used = false;
            return;
        }
        *static_cast<void**>(p) = free_[c];
        free_[c] = p;
    }

  private:
    static constexpr int kClasses = 16;               // 64 B << 0 .. 15
    static constexpr size_t kChunkBytes = (size_t)4 << 20;
    static int size_class(size_t bytes) {
        int c = 0;
        while (c < kClasses && ((size_t)64 << c) < bytes) ++c;
        return c < kClasses ? c : -1;
    }
    std::mutex mu_;
    void* free_[kClasses] = {};  // freed blocks per class, linked through their first word
    struct Big {
        void* p;
        size_t bytes;
        bool locked, used;
    };
    std::vector<std::pair<void*, bool>> chunks_;  // (memory, page-locked)
    std::vector<Big> big_;                        // blocks above 2 MiB, in use or kept for reuse
    uint8_t* cur_ = nullptr;
    size_t left_ = 0;
    int device_;
};

// Standard allocator over a HotPool.
template <class T>
struct HotAlloc {
    using value_type = T;
    HotPool* pool;
    explicit HotAlloc(HotPool* p) : pool(p) {}
    template <class U>
    HotAlloc(const HotAlloc<U>& o) : pool(o.pool) {}
    T* allocate(size_t n) {
        void* p = pool->allocate(n * sizeof(T));
        if (!p) throw std::bad_alloc();
        return static_cast<T*>(p);
    }
    void deallocate(T* p, size_t n) noexcept { pool->deallocate(p, n * sizeof(T)); }
    template <class U>
    bool operator==(const HotAlloc<U>& o) const { return pool == o.pool; }
    template <class U>
    bool operator!=(const HotAlloc<U>& o) const { return pool != o.pool; }
};

template <class T>
using HotVec = std::vector<T, HotAlloc<T>>;
template <class T>
using HotDeque = std::deque<T, HotAlloc<T>>;

// Page-locks the top of the calling thread's stack (where its frames and its
// thread-local data live) for the thread's life, so compaction cannot move
// those pages either.  No-op in a dry run or if the driver refuses.
class PinnedStackTop {
  public:
    explicit PinnedStackTop(bool page_locked) {
        if (!page_locked) return;
        pthread_attr_t attr;
        if (pthread_getattr_np(pthread_self(), &attr) != 0) return;
        void* addr = nullptr;
        size_t size = 0;
        const int rc = pthread_attr_getstack(&attr, &addr, &size);
        pthread_attr_destroy(&attr);
        if (rc != 0 || !addr || size < 2 * kPage) return;
        const uintptr_t lo = (uintptr_t)addr, hi = (lo + size) & ~(uintptr_t)(kPage - 1);
        const uintptr_t base = hi - std::min<uintptr_t>(kTop, hi - lo - kPage);
        if (cudaHostRegister((void*)base, hi - base, cudaHostRegisterDefault) == cudaSuccess) {
            base_ = (void*)base;
        } else {
            cudaGetLastError();
        }
    }
    ~PinnedStackTop() {
        if (base_) cudaHostUnregister(base_);
    }
    PinnedStackTop(const PinnedStackTop&) = delete;
    PinnedStackTop& operator=(const PinnedStackTop&) = delete;

  private:
    static constexpr uintptr_t kPage = 4096;
    static constexpr uintptr_t kTop = 256 << 10;
    void* base_ = nullptr;
};

// Completions waiting for aes_server_poll: a FIFO of fixed-size chunks.
// Chunks are made ahead of use (reserve: page-locked when a GPU is present, so
// the kernel's memory compaction cannot move them, and every page touched when
// made), and a chunk emptied by poll is kept for reuse.  Appending on the
// scheduler thread therefore normally calls no allocator and touches no page
// it has not touched before: a page fault there (a fresh page, or a page being
// migrated) can block for tens of milliseconds, and every thread waiting on the
// completion lock with it.  It grows without copying what it holds and
// releases from the front.
class CompletionFifo {
  public:
    static constexpr size_t kChunk = 16384;  // completions per chunk (640 KiB)

    CompletionFifo() = default;
    CompletionFifo(const CompletionFifo&) = delete;
    CompletionFifo& operator=(const CompletionFifo&) = delete;
    ~CompletionFifo() {
        for (Chunk* c : live_) drop(c);
        for (Chunk* c : spare_) drop(c);
    }

    void set_device(int device) { device_ = device; }  // page-locked chunks through this device; < 0: heap
    size_t size() const { return size_; }

    // Room for n more completions than are held now, made ahead of use.
    // Returns false when memory runs out (the FIFO still works: push then
    // allocates as it goes).
    bool reserve(size_t n) {
        const size_t free_in_tail = live_.empty() ? 0 : kChunk - tail_;
        size_t room = free_in_tail + kChunk * spare_.size();
        while (room < n) {
            Chunk* c = make(device_);
            if (!c) return false;
            spare_.push_back(c);
            room += kChunk;
        }
        const size_t chunks = live_.size() + spare_.size();
        if (live_.capacity() < chunks) live_.reserve(chunks);
        if (spare_.capacity() < chunks) spare_.reserve(chunks);
        return true;
    }

    // Appends n completions; returns how many were stored (fewer only when no
    // host memory is left for a chunk).
    size_t push(const aes_server_completion* c, size_t n) {
        const size_t n0 = n;
        while (n) {
            if (live_.empty() || tail_ == kChunk) {
                Chunk* k = nullptr;
                if (!spare_.empty()) {
                    k = spare_.back();
                    spare_.pop_back();
                } else {
                    k = make(-1);  // (no spare left: a plain allocation made here)
                    if (!k) return n0 - n;
                }
                live_.push_back(k);
                tail_ = 0;
            }
            const size_t m = std::min(n, kChunk - tail_);
            memcpy(live_.back()->e + tail_, c, m * sizeof(*c));
            tail_ += m;
            size_ += m;
            c += m;
            n -= m;
        }
        return n0;
    }

    // Moves up to max of the oldest completions to out; returns how many.
    size_t pop(aes_server_completion* out, size_t max) {
        size_t got = 0;
        while (got < max && size_) {
            const size_t end = live_.size() == 1 ? tail_ : kChunk;
            const size_t m = std::min(max - got, end - head_);
            memcpy(out + got, live_.front()->e + head_, m * sizeof(*out));
            head_ += m;
            got += m;
            size_ -= m;
            if (head_ == end) {
                if (live_.size() == 1) {  // empty: the chunk stays, refilled from its start
                    head_ = tail_ = 0;
                } else {
                    spare_.push_back(live_.front());
                    live_.erase(live_.begin());
                    head_ = 0;
                }
            }
        }
        return got;
    }

  private:
    struct Chunk {
        bool page_locked;
        aes_server_completion e[kChunk];
    };

    static Chunk* make(int device) {
        bool locked = false;
        Chunk* c = static_cast<Chunk*>(alloc_host(sizeof(Chunk), device, &locked));
        if (c) c->page_locked = locked;
        return c;
    }

    static void drop(Chunk* c) { free_host(c, c->page_locked); }

    std::vector<Chunk*> live_;   // oldest first; the last one is being filled
    std::vector<Chunk*> spare_;  // made ahead, or emptied by pop
    size_t head_ = 0;            // next to pop, in live_.front()
    size_t tail_ = 0;            // next free entry in live_.back()
    size_t size_ = 0;
    int device_ = -1;
};

// Completions made up front when a server starts, and kept spare beyond a
// replay's own requests when it starts.
constexpr size_t kCompletionsAhead = 4 * CompletionFifo::kChunk;

struct Slot {
    explicit Slot(HotPool* pool) : reqs(HotAlloc<Pending>(pool)) {}
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t* dev_buf = nullptr;
    uint8_t* host_buf = nullptr;
    HotVec<Pending> reqs;
    double launch_s = 0;
    uint64_t bytes = 0;
    bool busy = false;
};

// A request published to the resident kernel's ring.
struct ResItem {
    Pending p;
    uint64_t seq;         // request number in its direction, from 1
    uint32_t slot;        // its done counter on the device
    uint64_t first_tile;  // its tiles: [first_tile, first_tile + ntiles) of its direction
    uint64_t ntiles;
    uint64_t bytes;       // in+out bytes charged to the budget
    double launch_s;      // when it was published
    bool done;
};

// Scheduling diagnostics of one host thread, kept by that thread.  Every 16th
// pass, and on a pass that comes more than 50 us after the one before, it
// reads the thread's own CPU time and context-switch counts
// (getrusage(RUSAGE_THREAD)), closing a window.  The longest window in which
// the thread had work waiting throughout (it never slept on purpose) is kept
// with the CPU time the thread got in it and the involuntary switches
// (preemptions) it suffered: a window whose wall time far exceeds its CPU
// time, with involuntary switches, is time the thread was descheduled.
struct ThreadWatch {
    double win_start = 0, cpu_start = 0, prev_pass = 0;
    long invol_start = 0, vol_start = 0, minflt_start = 0, majflt_start = 0;
    bool win_busy = true, started = false;
    uint32_t passes = 0;
    uint64_t npasses = 0;
    double worst_wall = 0, worst_cpu = 0, worst_at = 0;
    long worst_invol = 0, worst_vol = 0, worst_minflt = 0, worst_majflt = 0, invol_total = 0, minflt_total = 0;

    static void usage(double* cpu, long* invol, long* vol = nullptr, long* minflt = nullptr, long* majflt = nullptr) {
        struct rusage u;
        memset(&u, 0, sizeof u);
        getrusage(RUSAGE_THREAD, &u);
        *cpu = (double)u.ru_utime.tv_sec + 1e-6 * u.ru_utime.tv_usec + (double)u.ru_stime.tv_sec +
               1e-6 * u.ru_stime.tv_usec;
        *invol = u.ru_nivcsw;
        if (vol) *vol = u.ru_nvcsw;
        if (minflt) *minflt = u.ru_minflt;
        if (majflt) *majflt = u.ru_majflt;
    }
    void sample(double now) {
        double cpu;
        long invol, vol, minflt, majflt;
        usage(&cpu, &invol, &vol, &minflt, &majflt);
        if (started) {
            invol_total += invol - invol_start;
            minflt_total += minflt - minflt_start;
            if (win_busy && now - win_start > worst_wall) {
                worst_wall = now - win_start;
                worst_cpu = cpu - cpu_start;
                worst_invol = invol - invol_start;
                worst_vol = vol - vol_start;
                worst_minflt = minflt - minflt_start;
                worst_majflt = majflt - majflt_start;
                worst_at = win_start;
            }
        }
        started = true;
        win_start = now;
        cpu_start = cpu;
        invol_start = invol;
        vol_start = vol;
        minflt_start = minflt;
        majflt_start = majflt;
        win_busy = true;
    }
    // A pass at `now`; busy: the thread had work waiting since its previous pass.
    void pass(double now, bool busy) {
        if (!started) sample(now);
        win_busy = win_busy && busy;
        const bool late = now - prev_pass > 50e-6;
        prev_pass = now;
        ++npasses;
        if (++passes % 16 == 0 || late) sample(now);
    }
};

}  // namespace gbaes

using namespace gbaes;

// Lives in page-locked memory itself (aes_server_create), like its hot containers.
struct aes_server {
    explicit aes_server(int host_device)
        : pool(host_device),
          keys(HotAlloc<aes_ctx>(&pool)),
          key_ptrs(HotAlloc<const aes_ctx*>(&pool)),
          inbox(HotAlloc<Pending>(&pool)),
          queue(HotAlloc<Pending>(&pool)),
          replay_reqs(HotAlloc<aes_server_request>(&pool)),
          replay_rc(HotAlloc<int32_t>(&pool)),
          rinflight{HotDeque<ResItem>(HotAlloc<ResItem>(&pool)), HotDeque<ResItem>(HotAlloc<ResItem>(&pool))} {}

    uint32_t magic = 0;
    aes_server_config cfg{};
    int device = 0;
    bool dryrun = false;
    HotPool pool;                       // the containers below allocate from it
    HotVec<aes_ctx> keys;               // host copies (key sizes, schedules)
    HotVec<const aes_ctx*> key_ptrs;
    uint4* dev_keys = nullptr;          // resident schedules: slot 2k = enc, 2k+1 = dec
    int* status = nullptr;
    size_t slot_cap = 0;
    std::vector<Slot> slots;
    std::chrono::steady_clock::time_point t0;

    std::mutex in_mu;
    std::condition_variable in_cv;  // wakes an idle scheduler
    HotVec<Pending> inbox;
    std::atomic<size_t> inbox_n{0};  // inbox.size(), readable without the lock
    std::vector<uint64_t> cancels;  // ids to cancel if still waiting for admission
    std::atomic<size_t> cancels_n{0};
    HotDeque<Pending> queue;  // scheduler thread only
    uint64_t inflight_bytes = 0;  // scheduler thread only
    uint64_t batch_counter = 0;   // scheduler thread only

    std::mutex out_mu;
    CompletionFifo done;  // completions waiting for aes_server_poll (under out_mu)
    std::atomic<uint64_t> lost_completions{0};  // not stored: no host memory left (aes_server_stats)

    std::mutex stats_mu;
    aes_server_stats stats{};

    std::atomic<uint64_t> submitted{0};
    std::atomic<uint64_t> finished{0};
    std::atomic<uint64_t> fault_batch{UINT64_MAX};
    std::atomic<bool> stop{false};
    std::atomic<bool> producer_stop{false};
    std::atomic<bool> producer_running{false};
    std::thread scheduler;
    std::thread producer;
    HotVec<aes_server_request> replay_reqs;
    HotVec<int32_t> replay_rc;  // each replayed request's check, made when the replay starts
    double replay_start = 0;

    // Resident mode (scheduler thread only, except where noted).
    bool resident = false;
    uint32_t tile_blocks = 0;     // a tile's capacity: threads * blocks_per_thread
    uint32_t spread = 1;          // CTAs of the resident kernel
    uint64_t rtiles_open = 0;     // tiles of published, unfinished requests
    uint8_t* ring_mem = nullptr;  // page-locked and mapped (plain host memory in a dry run)
    ResCtrl* rctrl = nullptr;     // host views into ring_mem
    ResTile* rtiles = nullptr;
    ResDone* rcq = nullptr;       // completion queue (host view)
    uint64_t rcq_head = 0;        // completions consumed
    ResArgs rargs{};              // device views
    cudaStream_t rstream = nullptr;
    uint64_t rpub[2] = {0, 0};        // tiles published per direction
    uint64_t ritems[2] = {0, 0};      // requests published per direction
    uint64_t rrel_tiles[2] = {0, 0};  // tiles below this are finished: their ring slots are free
    uint64_t rrel_items[2] = {0, 0};  // requests up to this sequence number are finished
    HotDeque<ResItem> rinflight[2];
    bool rlive = false;               // a kernel (or its dry-run stand-in) is running
    bool rstopping = false;           // its stop word is set: nothing is published until it has ended
    double rstop_s = 0;               // when the stop word was set
    double rprogress_s = 0;           // last publication or completion
    uint64_t rgen = 0;                // launches so far (the running kernel's number)
    uint32_t rgrid = 0;               // its CTAs
    uint64_t* rexit = nullptr;        // host view of the CTAs' exit words
    double rlaunch_s = 0;             // its launch
    // Dry run: one host thread runs the kernel's ticket/record/count/status protocol.
    std::vector<uint64_t> fake_claim, fake_done;  // stand-in thread, or the scheduler while none runs
    uint64_t fake_cq_next = 0;
    std::vector<uint64_t> fake_abandon[2];
    std::thread fake;
    std::atomic<bool> fake_running{false};

    // Host-thread diagnostics (aes_server_stats): the scheduler's, kept by the
    // scheduler thread; the replay thread's, kept by that thread.
    ThreadWatch sched_watch;
    double lock_wait_max[3] = {0, 0, 0}, lock_wait_at[3] = {0, 0, 0};  // submissions, completions, stats
    double cuda_call_max = 0, cuda_call_at = 0;
    uint64_t stream_queries[2] = {0, 0};  // resident: to confirm an end, for lack of progress
    double phase_max[5] = {0, 0, 0, 0, 0}, phase_at[5] = {0, 0, 0, 0, 0};  // scheduler pass phases
    double inbox_hold_max = 0;                 // by the scheduler
    std::atomic<uint64_t> submit_hold_ns{0};   // by a submitter (replay thread or aes_server_submit)
    aes_server_diag diag{};       // published copy (stats_mu)
    int sched_cpu = -1, producer_cpu = -1;  // CPU each thread is pinned to (AES_SERVER_PIN_THREADS), or -1
    bool sched_slept = false;     // scheduler: its last idle wait slept on the condition variable
    bool self_locked = false;     // this object's own memory is page-locked

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace gbaes {

// A lock taken by the scheduler thread on a mutex that other threads share;
// the wait counts toward the scheduler's longest wait for that lock.
enum { kLockInbox = 0, kLockDone = 1, kLockStats = 2 };

class SchedLock {
   public:
    SchedLock(aes_server* S, int which)
        : m_(which == kLockInbox ? S->in_mu : which == kLockDone ? S->out_mu : S->stats_mu) {
        const auto t = std::chrono::steady_clock::now();
        m_.lock();
        const double w = std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count();
        if (w > S->lock_wait_max[which]) {
            S->lock_wait_max[which] = w;
            S->lock_wait_at[which] = S->now();
        }
    }
    ~SchedLock() { m_.unlock(); }
    SchedLock(const SchedLock&) = delete;
    SchedLock& operator=(const SchedLock&) = delete;

   private:
    std::mutex& m_;
};

// Times one CUDA call of the scheduler thread.
template <class F>
static auto timed_cuda(aes_server* S, F&& f) -> decltype(f()) {
    const double t = S->now();
    auto r = f();
    const double d = S->now() - t;
    if (d > S->cuda_call_max) {
        S->cuda_call_max = d;
        S->cuda_call_at = t;
    }
    return r;
}

// Scheduler pass phases: 0 submissions, 1 completions, 2 kernel or event
// queries, 3 admission, 4 launch and statistics.  Ends phase i begun at *t.
enum { kPhaseInbox = 0, kPhaseDone = 1, kPhaseQuery = 2, kPhaseAdmit = 3, kPhaseLaunch = 4 };

static void end_phase(aes_server* S, int i, double* t) {
    const double now = S->now();
    if (now - *t > S->phase_max[i]) {
        S->phase_max[i] = now - *t;
        S->phase_at[i] = *t;
    }
    *t = now;
}

// Pins the calling thread to one CPU of the process's affinity set: the
// last (which = 0) or the one before it (which = 1).  Returns the CPU or -1.
static int pin_thread(int which) {
    cpu_set_t set;
    CPU_ZERO(&set);
    if (sched_getaffinity(0, sizeof set, &set) != 0) return -1;
    int found = 0;
    for (int c = CPU_SETSIZE - 1; c >= 0; --c) {
        if (!CPU_ISSET(c, &set)) continue;
        if (found++ < which) continue;
        cpu_set_t one;
        CPU_ZERO(&one);
        CPU_SET(c, &one);
        return pthread_setaffinity_np(pthread_self(), sizeof one, &one) == 0 ? c : -1;
    }
    return -1;
}

// Copies the scheduler's diagnostics into the published copy (caller holds stats_mu).
static void publish_diagnostics(aes_server* S) {
    const ThreadWatch& w = S->sched_watch;
    aes_server_diag& d = S->diag;
    d.sched_passes = w.npasses;
    d.sched_worst_window_ns = (uint64_t)(1e9 * w.worst_wall);
    d.sched_worst_window_cpu_ns = (uint64_t)(1e9 * w.worst_cpu);
    d.sched_worst_window_invol = (uint64_t)w.worst_invol;
    d.sched_worst_window_vol = (uint64_t)w.worst_vol;
    d.sched_worst_window_at_ns = (uint64_t)(1e9 * w.worst_at);
    d.sched_worst_window_minflt = (uint64_t)w.worst_minflt;
    d.sched_worst_window_majflt = (uint64_t)w.worst_majflt;
    d.sched_invol = (uint64_t)w.invol_total;
    d.sched_minflt = (uint64_t)w.minflt_total;
    for (int i = 0; i < 3; ++i) {
        d.lock_wait_max_ns[i] = (uint64_t)(1e9 * S->lock_wait_max[i]);
        d.lock_wait_at_ns[i] = (uint64_t)(1e9 * S->lock_wait_at[i]);
    }
    d.cuda_call_max_ns = (uint64_t)(1e9 * S->cuda_call_max);
    d.cuda_call_at_ns = (uint64_t)(1e9 * S->cuda_call_at);
    d.stream_queries[0] = S->stream_queries[0];
    d.stream_queries[1] = S->stream_queries[1];
    for (int i = 0; i < 5; ++i) {
        d.sched_phase_max_ns[i] = (uint64_t)(1e9 * S->phase_max[i]);
        d.sched_phase_at_ns[i] = (uint64_t)(1e9 * S->phase_at[i]);
    }
    d.inbox_hold_max_ns[0] = (uint64_t)(1e9 * S->inbox_hold_max);
    d.inbox_hold_max_ns[1] = S->submit_hold_ns.load(std::memory_order_relaxed);
    d.sched_cpu = S->sched_cpu;
}

static void complete(aes_server* S, HotVec<Pending>& reqs, int status, double launch_s, double done_s) {
    {
        SchedLock lk(S, kLockDone);
        for (const Pending& p : reqs) {
            aes_server_completion c;
            c.id = p.r.id;
            c.status = status;
            c.batch_msgs = (uint32_t)reqs.size();
            c.arrival_s = p.arrival;
            c.launch_s = launch_s;
            c.done_s = done_s;
            if (S->done.push(&c, 1) != 1) S->lost_completions.fetch_add(1);
        }
    }
    {
        SchedLock lk(S, kLockStats);
        S->stats.completed += reqs.size();
        if (status != AES_OK) S->stats.failed += reqs.size();
    }
    S->finished.fetch_add(reqs.size());
    reqs.clear();
}

static uint64_t request_bytes(const aes_server_request& r) { return 32ull * r.nblocks; }

// Launches one micro-batch on a free slot.  Returns AES_OK or the error with
// which the batch's requests are completed.
static int launch_slot(aes_server* S, Slot& slot) {
    const uint64_t index = S->batch_counter++;
    if (index == S->fault_batch.load()) return fail(AES_ERR_DEVICE, "injected fault on batch %llu", (unsigned long long)index);
    if (S->dryrun) return AES_OK;
    std::vector<aes_msg_desc> d(slot.reqs.size());
    for (size_t i = 0; i < slot.reqs.size(); ++i) {
        const aes_server_request& r = slot.reqs[i].r;
        d[i].in_off = (uint64_t)(uintptr_t)r.in;  // absolute addresses: the kernel's base pointers are 0
        d[i].out_off = (uint64_t)(uintptr_t)r.out;
        d[i].nblocks = r.nblocks;
        d[i].key_index = r.key_index;
        d[i].decrypt = r.decrypt;
    }
    HostPlan H;
    const uint32_t tb = 32u * (uint32_t)S->cfg.blocks_per_thread;  // one pass per warp tile: low latency
    int rc = build_host_plan(d.data(), d.size(), S->key_ptrs.data(), S->key_ptrs.size(), tb, false, &H);
    if (rc) return rc;
    if (H.ntiles == 0) return AES_OK;
    const size_t off_msgs = 256;
    const size_t off_tiles = off_msgs + ((H.msgs.size() * sizeof(MsgDev) + 255) & ~(size_t)255);
    const size_t bytes = off_tiles + H.tile_msg.size() * 4 + 4;
    if (bytes > S->slot_cap) return fail(AES_ERR_ARG, "batch tables (%zu B) exceed the slot (%zu B)", bytes, S->slot_cap);
    memset(slot.host_buf, 0, 256);
    memcpy(slot.host_buf + off_msgs, H.msgs.data(), H.msgs.size() * sizeof(MsgDev));
    memcpy(slot.host_buf + off_tiles, H.tile_msg.data(), H.tile_msg.size() * 4);
    cudaError_t e = cudaMemcpyAsync(slot.dev_buf, slot.host_buf, bytes, cudaMemcpyHostToDevice, slot.stream);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "batch table upload: %s", cudaGetErrorString(e));
    BatchArgs a;
    memset(&a, 0, sizeof a);
    a.in = nullptr;
    a.out = nullptr;
    a.msgs = (const MsgDev*)(slot.dev_buf + off_msgs);
    a.keys = S->dev_keys;
    a.tile_msg = (const uint32_t*)(slot.dev_buf + off_tiles);
    a.counter = (unsigned*)slot.dev_buf;
    a.status = S->status;
    a.ntiles = H.ntiles;
    a.tile_blocks = H.tile_blocks;
    memcpy(a.groups, H.groups, sizeof a.groups);
    rc = launch_batch_kernel(a, S->cfg.threads, S->cfg.blocks_per_thread, slot.stream);
    if (rc) return rc;
    e = cudaEventRecord(slot.done, slot.stream);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "batch event: %s", cudaGetErrorString(e));
    return AES_OK;
}

// Moves new submissions into the admission queue and completes cancelled
// requests that are still waiting there.  Returns true if anything changed.
static bool take_inbox(aes_server* S) {
    bool worked = false;
    std::vector<uint64_t> cancels;
    if (S->inbox_n.load(std::memory_order_acquire) == 0 && !S->cancels_n.load(std::memory_order_acquire))
        return false;  // nothing new: leave the lock to the producers
    {
        SchedLock lk(S, kLockInbox);
        const double t = S->now();
        if (!S->inbox.empty()) {
            for (Pending& p : S->inbox) S->queue.push_back(p);
            S->inbox.clear();
            S->inbox_n.store(0, std::memory_order_release);
            worked = true;
        }
        cancels.swap(S->cancels);
        S->cancels_n.store(0, std::memory_order_release);
        S->inbox_hold_max = std::max(S->inbox_hold_max, S->now() - t);
    }
    if (!cancels.empty()) {  // only requests not yet admitted can be cancelled
        HotVec<Pending> gone(HotAlloc<Pending>(&S->pool));
        for (auto it = S->queue.begin(); it != S->queue.end();) {
            if (std::find(cancels.begin(), cancels.end(), it->r.id) != cancels.end()) {
                gone.push_back(*it);
                it = S->queue.erase(it);
            } else {
                ++it;
            }
        }
        if (!gone.empty()) {
            const double t = S->now();
            complete(S, gone, AES_ERR_STATE, t, t);
            worked = true;
        }
    }
    return worked;
}

// Sleeps until a submission, a cancellation or shutdown when nothing is queued
// or in flight (bounded, so a missed wake-up costs 1 ms); yields otherwise.
// Returns false when the scheduler should exit.
static bool idle_wait(aes_server* S, bool idle) {
    if (!idle) {
        std::this_thread::yield();
        return true;
    }
    S->sched_slept = true;  // (the scheduler's next pass closes no "busy" window)
    std::unique_lock<std::mutex> lk(S->in_mu);
    if (S->inbox.empty() && S->cancels.empty() && S->stop.load()) return false;
    S->in_cv.wait_for(lk, std::chrono::milliseconds(1),
                      [S] { return !S->inbox.empty() || !S->cancels.empty() || S->stop.load(); });
    return true;
}

static void scheduler_main(aes_server* S) {
    if (!S->dryrun) cudaSetDevice(S->device);
    pthread_setname_np(pthread_self(), "gbaes-sched");  // (names for ps, top and /proc/<pid>/task)
    const PinnedStackTop stack_top(!S->dryrun);
    if (S->cfg.flags & AES_SERVER_PIN_THREADS) S->sched_cpu = pin_thread(0);
    for (;;) {
        S->sched_watch.pass(S->now(), !S->sched_slept);
        S->sched_slept = false;
        double ph = S->now();
        bool worked = take_inbox(S);
        end_phase(S, kPhaseInbox, &ph);
        // Completions.
        for (Slot& slot : S->slots) {
            if (!slot.busy) continue;
            int st = AES_OK;
            if (S->dryrun) {
                if (S->now() - slot.launch_s < 1e-6 * S->cfg.dryrun_batch_us) continue;
            } else {
                cudaError_t q = timed_cuda(S, [&] { return cudaEventQuery(slot.done); });
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) st = AES_ERR_CUDA;
            }
            const double t = S->now();
            S->inflight_bytes -= slot.bytes;
            slot.bytes = 0;
            slot.busy = false;
            complete(S, slot.reqs, st, slot.launch_s, t);
            worked = true;
        }
        end_phase(S, kPhaseQuery, &ph);  // (event queries and completions)
        // Admission in arrival order, then launch on free slots.
        for (Slot& slot : S->slots) {
            if (slot.busy || S->queue.empty()) continue;
            uint64_t blocks = 0, bytes = 0;
            while (!S->queue.empty() && slot.reqs.size() < S->cfg.max_batch_msgs) {
                const Pending& p = S->queue.front();
                const uint64_t b = request_bytes(p.r);
                if (S->inflight_bytes + bytes + b > S->cfg.budget_bytes) break;
                if (!slot.reqs.empty() && blocks + p.r.nblocks > S->cfg.max_batch_blocks) break;
                blocks += p.r.nblocks;
                bytes += b;
                slot.reqs.push_back(p);
                S->queue.pop_front();
            }
            if (slot.reqs.empty()) break;  // the budget is full: wait for completions
            slot.launch_s = S->now();
            int rc = timed_cuda(S, [&] { return launch_slot(S, slot); });
            if (rc != AES_OK && !S->dryrun) cudaStreamSynchronize(slot.stream);  // staging may still be read
            {
                SchedLock lk(S, kLockStats);
                S->stats.batches++;
                S->stats.max_batch_msgs = std::max<uint64_t>(S->stats.max_batch_msgs, slot.reqs.size());
            }
            if (rc != AES_OK) {
                complete(S, slot.reqs, rc, slot.launch_s, S->now());
            } else {
                slot.busy = true;
                slot.bytes = bytes;
                S->inflight_bytes += bytes;
                SchedLock lk(S, kLockStats);
                S->stats.max_inflight_bytes = std::max<uint64_t>(S->stats.max_inflight_bytes, S->inflight_bytes);
            }
            worked = true;
        }
        end_phase(S, kPhaseLaunch, &ph);  // (admission and launches)
        {
            SchedLock lk(S, kLockStats);
            S->stats.max_queue = std::max<uint64_t>(S->stats.max_queue, S->queue.size());
            publish_diagnostics(S);
        }
        if (!worked) {
            bool idle = S->queue.empty();
            for (const Slot& slot : S->slots) idle = idle && !slot.busy;
            if (!idle_wait(S, idle)) break;  // batches in flight: poll their events
        }
    }
}

// ------------------------------------------------------------ resident mode

// Dry-run stand-in for the resident kernel: one host thread follows the
// kernel's ticket protocol (a ticket always held in its own direction, one in
// the other when that has untaken published tiles; own direction first unless
// the other's tile has waited 20 us), "enciphers" each tile for
// dryrun_batch_us, counts blocks per request, publishes completions, and on
// the stop word or its lifetime leaves, writing held tickets to the abandon
// list (and, like a kernel whose last CTAs are still finishing, counting as
// running for another 0.5 ms).
static void fake_kernel_main(aes_server* S) {
    using clock = std::chrono::steady_clock;
    const clock::time_point start = clock::now();
    const uint32_t rt = S->rargs.ring_tiles, ri = S->rargs.ring_items;
    constexpr uint64_t kNone = ~0ull;
    uint64_t held[2] = {kNone, kNone};
    clock::time_point ready[2];  // first seen published
    bool seen[2] = {false, false};
    int dir = 0;
    for (;;) {
        uint64_t pub[2] = {__atomic_load_n(&S->rctrl->pub[0], __ATOMIC_ACQUIRE),
                           __atomic_load_n(&S->rctrl->pub[1], __ATOMIC_ACQUIRE)};
        const int oth = dir ^ 1;
        if (held[dir] == kNone) {
            held[dir] = S->fake_claim[dir]++;
            seen[dir] = false;
        }
        if (held[oth] == kNone && S->fake_claim[oth] < pub[oth]) {
            held[oth] = S->fake_claim[oth]++;
            seen[oth] = false;
        }
        const clock::time_point t = clock::now();
        bool ok[2];
        for (int d = 0; d < 2; ++d) {
            ok[d] = held[d] != kNone && held[d] < pub[d];
            if (ok[d] && !seen[d]) {
                seen[d] = true;
                ready[d] = t;
            }
        }
        int got = -1;  // own direction first, unless the other's tile has waited 20 us
        if (ok[oth] && (!ok[dir] || t - ready[oth] > std::chrono::microseconds(20)))
            got = oth;
        else if (ok[dir])
            got = dir;
        if (got < 0) {
            const bool expired = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clock::now() - start)
                                     .count() > S->rargs.lifetime_ns;
            if (__atomic_load_n(&S->rctrl->stop, __ATOMIC_ACQUIRE) || expired) {
                bool published = false;
                for (int d = 0; d < 2; ++d)
                    published = published ||
                                (held[d] != kNone && held[d] < __atomic_load_n(&S->rctrl->pub[d], __ATOMIC_ACQUIRE));
                if (published) continue;
                for (int d = 0; d < 2; ++d)
                    if (held[d] != kNone) S->fake_abandon[d].push_back(held[d]);
                // The kernel's CTAs leave one by one: the kernel still runs for
                // a while after the first have abandoned their tickets, and the
                // scheduler may publish those tiles meanwhile.
                std::this_thread::sleep_for(std::chrono::microseconds(500));
                break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            continue;
        }
        dir = got;
        const ResTile R = S->rtiles[(uint64_t)got * rt + (held[got] & (rt - 1))];
        held[got] = kNone;
        seen[got] = false;
        if (S->cfg.dryrun_batch_us) std::this_thread::sleep_for(std::chrono::microseconds(S->cfg.dryrun_batch_us));
        uint64_t& done = S->fake_done[(uint64_t)got * ri + R.item];
        done += R.nblocks;
        if (done == R.item_blocks) {
            done = 0;
            const uint64_t i = S->fake_cq_next++;
            __atomic_store_n(&S->rcq[i & (S->rargs.cq_size - 1)].word, cq_word(i, S->rargs.cq_log2, got, R.seq),
                             __ATOMIC_RELEASE);
        }
    }
    S->fake_running.store(false, std::memory_order_release);
}

// Starts the kernel (or its dry-run stand-in).
static int start_resident(aes_server* S) {
    S->rlaunch_s = S->now();
    if (S->dryrun) {
        if (S->fake.joinable()) S->fake.join();  // the previous one has finished
        S->fake_running.store(true);
        S->fake = std::thread(fake_kernel_main, S);
        return AES_OK;
    }
    S->rargs.gen = ++S->rgen;
    return launch_resident(S->rargs, S->cfg.threads, S->cfg.blocks_per_thread, S->rstream);
}

// True while the kernel runs; AES_ERR_CUDA in *err if it failed.
// True while the kernel runs; AES_ERR_CUDA in *err if it failed.  While its
// CTAs keep working this makes no CUDA call: each CTA marks its normal exit in
// page-locked memory, and the stream is asked only to confirm an end that every
// CTA has marked, or when the kernel shows no sign of life (`suspect`: nothing
// published or completed for 50 ms with work in flight, or 50 ms after the stop
// word), which is how a fault shows.  (Asked every 50 us, the stream query now
// and then waited tens of milliseconds inside the driver, and every request in
// flight waited with it.)
static bool resident_running(aes_server* S, int* err, bool suspect) {
    *err = AES_OK;
    if (S->dryrun) return S->fake_running.load(std::memory_order_acquire);
    bool all = true;
    for (uint32_t i = 0; i < S->rgrid && all; ++i) all = __atomic_load_n(&S->rexit[i], __ATOMIC_ACQUIRE) == S->rgen;
    if (!all && !suspect) return true;
    ++S->stream_queries[all ? 0 : 1];
    const cudaError_t q = timed_cuda(S, [&] { return cudaStreamQuery(S->rstream); });
    if (q == cudaErrorNotReady) return true;
    if (q != cudaSuccess) *err = fail(AES_ERR_CUDA, "resident kernel: %s", cudaGetErrorString(q));
    return false;
}

// After a kernel has ended: re-publishes every abandoned ticket whose tile had
// been published (nobody enciphered it), moves each ticket counter back to the
// first tile nobody took (tickets taken ahead of publication are void), and
// clears the abandon list and the stop word for the next kernel.
static int recover_resident(aes_server* S) {
    const uint32_t rt = S->rargs.ring_tiles;
    unsigned long long claim[2] = {0, 0}, n[2] = {0, 0};
    std::vector<unsigned long long> ab(2 * (size_t)kAbandonCap, 0);
    if (S->dryrun) {
        if (S->fake.joinable()) S->fake.join();
        for (int d = 0; d < 2; ++d) {
            claim[d] = S->fake_claim[d];
            n[d] = S->fake_abandon[d].size();
            for (size_t i = 0; i < S->fake_abandon[d].size() && i < kAbandonCap; ++i)
                ab[(size_t)d * kAbandonCap + i] = S->fake_abandon[d][i];
        }
    } else {  // on the kernel's own stream: other streams' work does not delay the recovery
        cudaStream_t st = S->rstream;
        cudaError_t e = cudaMemcpyAsync(claim, S->rargs.claim, sizeof claim, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(n, S->rargs.abandon_n, sizeof n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ab.data(), S->rargs.abandon, ab.size() * sizeof(ab[0]), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(AES_ERR_CUDA, "resident recovery: %s", cudaGetErrorString(e));
    }
    for (int d = 0; d < 2; ++d) {
        if (n[d] > kAbandonCap) return fail(AES_ERR_DEVICE, "resident kernel: abandon list overflowed");
        const uint64_t pub = S->rpub[d];
        claim[d] = std::min<unsigned long long>(claim[d], pub);
        for (unsigned long long i = 0; i < n[d]; ++i) {
            const uint64_t t = ab[(size_t)d * kAbandonCap + i];
            if (t >= pub) continue;  // never published: void
            if (S->rpub[d] + 1 - S->rrel_tiles[d] > rt) return fail(AES_ERR_STATE, "resident ring full during recovery");
            S->rtiles[(uint64_t)d * rt + (S->rpub[d] & (rt - 1))] = S->rtiles[(uint64_t)d * rt + (t & (rt - 1))];
            ++S->rpub[d];
            std::lock_guard<std::mutex> lk(S->stats_mu);
            S->stats.recovered_tiles++;
        }
        __atomic_store_n(&S->rctrl->pub[d], S->rpub[d], __ATOMIC_RELEASE);
    }
    if (S->dryrun) {
        for (int d = 0; d < 2; ++d) {
            S->fake_claim[d] = claim[d];
            S->fake_abandon[d].clear();
        }
    } else {
        const unsigned long long zero[2] = {0, 0};
        cudaStream_t st = S->rstream;
        cudaError_t e = cudaMemcpyAsync(S->rargs.claim, claim, sizeof claim, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S->rargs.abandon_n, zero, sizeof zero, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // (the sources live on this stack)
        if (e != cudaSuccess) return fail(AES_ERR_CUDA, "resident recovery: %s", cudaGetErrorString(e));
    }
    __atomic_store_n(&S->rctrl->stop, 0u, __ATOMIC_RELEASE);
    return AES_OK;
}

// Completes every published, unfinished request with `status` (the kernel has
// failed or could not start: their work will not be done), frees their ring
// space and moves the ticket counters past their tiles, so that a later kernel
// starts with the next request.  Called only while no kernel runs.
static void fail_resident_inflight(aes_server* S, int status) {
    const double t = S->now();
    for (int d = 0; d < 2; ++d) {
        for (ResItem& it : S->rinflight[d]) {
            if (it.done) continue;
            HotVec<Pending> one(1, it.p, HotAlloc<Pending>(&S->pool));
            S->inflight_bytes -= it.bytes;
            complete(S, one, status, it.launch_s, t);
        }
        S->rinflight[d].clear();
        S->rrel_tiles[d] = S->rpub[d];
        S->rrel_items[d] = S->ritems[d];
    }
    S->rtiles_open = 0;
    if (S->dryrun) {
        for (int d = 0; d < 2; ++d) {
            S->fake_claim[d] = S->rpub[d];
            S->fake_abandon[d].clear();
        }
        std::fill(S->fake_done.begin(), S->fake_done.end(), 0);
    } else {
        unsigned long long claim[2] = {S->rpub[0], S->rpub[1]};
        const unsigned long long zero[2] = {0, 0};
        cudaStream_t st = S->rstream;
        cudaMemcpyAsync(S->rargs.claim, claim, sizeof claim, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(S->rargs.abandon_n, zero, sizeof zero, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(S->rargs.done, 0, sizeof(unsigned long long) * 2 * S->rargs.ring_items, st);
        cudaStreamSynchronize(st);
        cudaGetLastError();
    }
    __atomic_store_n(&S->rctrl->stop, 0u, __ATOMIC_RELEASE);
}

constexpr uint64_t kMinSplitBlocks = 256;  // below this, splitting a request costs more than it saves

// Blocks per tile for a request of n blocks: spread over the CTAs that have
// nothing to do (the CTA count minus the tiles of unfinished requests; a
// tile's rounds are bound by its SM's shared-memory lookups, so smaller tiles
// on idle SMs finish sooner), but no smaller than kMinSplitBlocks and no
// larger than a tile's capacity.  Under load the CTAs are busy and requests go
// out in whole tiles (splitting then only adds per-tile overhead).  Tiles per
// request: at most max(spread, ceil(n / capacity)).
static uint64_t request_tile_blocks(const aes_server* S, uint64_t n) {
    const uint64_t cap = S->tile_blocks;
    const uint64_t lo = std::min<uint64_t>(kMinSplitBlocks, cap);
    const uint64_t idle = S->rtiles_open < S->spread ? S->spread - S->rtiles_open : 1;
    return std::min<uint64_t>(cap, std::max<uint64_t>(lo, (n + idle - 1) / idle));
}

// Writes request p as tile records and publishes them.  Returns false if the
// direction's ring has no room for it now.
static bool publish(aes_server* S, const Pending& p, uint64_t bytes, double now) {
    const int d = (int)p.r.decrypt;
    const uint32_t rt = S->rargs.ring_tiles, ri = S->rargs.ring_items;
    const uint64_t tb = request_tile_blocks(S, p.r.nblocks);
    const uint64_t ntiles = (p.r.nblocks + tb - 1) / tb;
    if (S->rpub[d] + ntiles - S->rrel_tiles[d] > rt || S->ritems[d] - S->rrel_items[d] >= ri) return false;
    const uint64_t seq = ++S->ritems[d];
    const uint32_t slot = (uint32_t)((seq - 1) & (ri - 1));
    const aes_ctx& key = S->keys[p.r.key_index];
    for (uint64_t j = 0; j < ntiles; ++j) {
        ResTile& R = S->rtiles[(uint64_t)d * rt + ((S->rpub[d] + j) & (rt - 1))];
        R.in = (uint64_t)(uintptr_t)p.r.in + 16 * tb * j;
        R.out = (uint64_t)(uintptr_t)p.r.out + 16 * tb * j;
        R.item_blocks = p.r.nblocks;
        R.seq = seq;
        R.nblocks = (uint32_t)std::min<uint64_t>(tb, p.r.nblocks - tb * j);
        R.key_slot = 2u * p.r.key_index + (uint32_t)d;
        R.item = slot;
        R.nr = (uint32_t)key.nr;
    }
    ResItem it{p, seq, slot, S->rpub[d], ntiles, bytes, now, false};
    S->rpub[d] += ntiles;
    S->rtiles_open += ntiles;
    __atomic_store_n(&S->rctrl->pub[d], S->rpub[d], __ATOMIC_RELEASE);  // records before the count
    S->rinflight[d].push_back(it);
    return true;
}

static void scheduler_resident(aes_server* S) {
    if (!S->dryrun) cudaSetDevice(S->device);
    pthread_setname_np(pthread_self(), "gbaes-sched");  // (names for ps, top and /proc/<pid>/task)
    const PinnedStackTop stack_top(!S->dryrun);
    if (S->cfg.flags & AES_SERVER_PIN_THREADS) S->sched_cpu = pin_thread(0);
    double last_work = S->now(), last_query = 0;
    HotVec<aes_server_completion> finished(HotAlloc<aes_server_completion>(&S->pool));
    const double idle_s = 1e-6 * S->cfg.resident_idle_us;
    // Normally well before the kernel's own bound (80%); later in tests of the recovery.
    const double restart_s = 1e-5 * S->cfg.resident_restart_pct * S->cfg.resident_lifetime_ms;
    for (;;) {
        double ph = S->now();
        bool worked = take_inbox(S);
        end_phase(S, kPhaseInbox, &ph);
        // Completions: new entries of the completion queue, in order.  Ring
        // space is freed in publication order (a request's tiles and slot are
        // reused only once it and every request before it in its direction
        // have finished).
        finished.clear();
        const double pass_s = S->now();  // one clock read per pass, not per request
        S->sched_watch.pass(pass_s, !S->sched_slept);
        S->sched_slept = false;
        for (;;) {
            const ResDone* e = &S->rcq[S->rcq_head & (S->rargs.cq_size - 1)];
            const uint64_t w = __atomic_load_n(&e->word, __ATOMIC_ACQUIRE);
            if ((w >> 40) != cq_lap(S->rcq_head, S->rargs.cq_log2)) break;  // not written in this lap yet
            ++S->rcq_head;
            const int d = (int)((w >> 39) & 1u);
            HotDeque<ResItem>& q = S->rinflight[d];
            if (q.empty()) continue;  // (not in flight)
            const uint64_t seq = q.front().seq + (((w & kCqSeqMask) - q.front().seq) & kCqSeqMask);
            if (seq - q.front().seq >= q.size()) continue;  // (not in flight)
            ResItem& it = q[seq - q.front().seq];
            if (it.done) continue;
            it.done = true;
            S->inflight_bytes -= it.bytes;
            S->rtiles_open -= it.ntiles;
            finished.push_back(aes_server_completion{it.p.r.id, AES_OK, 1, it.p.arrival, it.launch_s, pass_s});
            S->rprogress_s = pass_s;
        }
        for (int d = 0; d < 2; ++d) {
            while (!S->rinflight[d].empty() && S->rinflight[d].front().done) {
                const ResItem& f = S->rinflight[d].front();
                S->rrel_tiles[d] = f.first_tile + f.ntiles;
                S->rrel_items[d] = f.seq;
                S->rinflight[d].pop_front();
            }
        }
        if (!finished.empty()) {  // one hand-over per pass, not one per request
            {
                SchedLock lk(S, kLockDone);
                const size_t kept = S->done.push(finished.data(), finished.size());
                if (kept != finished.size()) S->lost_completions.fetch_add(finished.size() - kept);
            }
            {
                SchedLock lk(S, kLockStats);
                S->stats.completed += finished.size();
            }
            S->finished.fetch_add(finished.size());
            worked = true;
        }
        end_phase(S, kPhaseDone, &ph);
        // Has the kernel ended?  (Its CTAs' exit words: on every pass while it
        // is stopping, else every 50 us -- it ends on its own only at its
        // lifetime bound or on a fault.)
        if (S->rlive && (S->rstopping || pass_s - last_query > 50e-6)) {
            last_query = pass_s;
            int err = AES_OK;
            const bool busy = !S->rinflight[0].empty() || !S->rinflight[1].empty();
            const bool suspect = (busy && pass_s - S->rprogress_s > 0.05) || (S->rstopping && pass_s - S->rstop_s > 0.05);
            if (!resident_running(S, &err, suspect)) {
                S->rlive = false;
                S->rstopping = false;
                if (err == AES_OK) err = recover_resident(S);
                if (err != AES_OK) fail_resident_inflight(S, err);
                worked = true;
            }
        }
        bool inflight = !S->rinflight[0].empty() || !S->rinflight[1].empty();
        // Stop the kernel (no publishing until it has ended) when the server
        // has been idle, or before the kernel reaches its lifetime bound.
        const bool quiet = !inflight && S->queue.empty();
        if (S->rlive && !S->rstopping &&
            ((quiet && (S->now() - last_work > idle_s || S->stop.load())) || S->now() - S->rlaunch_s > restart_s)) {
            __atomic_store_n(&S->rctrl->stop, 1u, __ATOMIC_RELEASE);
            S->rstopping = true;
            S->rstop_s = S->now();
        }
        end_phase(S, kPhaseQuery, &ph);
        // Admission in arrival order while the budget and the ring have room.
        const double admit_s = S->now();
        size_t admitted = 0;
        while (!S->rstopping && !S->queue.empty()) {
            const Pending& p = S->queue.front();
            const uint64_t b = request_bytes(p.r);
            if (p.r.nblocks == 0) {
                HotVec<Pending> one(1, p, HotAlloc<Pending>(&S->pool));
                S->queue.pop_front();
                const double t = S->now();
                complete(S, one, AES_OK, t, t);
                worked = true;
                continue;
            }
            if (S->inflight_bytes + b > S->cfg.budget_bytes) break;
            if (S->batch_counter == S->fault_batch.load()) {
                ++S->batch_counter;
                HotVec<Pending> one(1, p, HotAlloc<Pending>(&S->pool));
                S->queue.pop_front();
                const double t = S->now();
                complete(S, one, fail(AES_ERR_DEVICE, "injected fault"), t, t);
                worked = true;
                continue;
            }
            if (!publish(S, p, b, admit_s)) break;
            S->rprogress_s = admit_s;
            ++S->batch_counter;
            S->inflight_bytes += b;
            S->queue.pop_front();
            ++admitted;
            worked = true;
        }
        end_phase(S, kPhaseAdmit, &ph);
        {
            SchedLock lk(S, kLockStats);
            if (admitted) {
                S->stats.max_inflight_bytes = std::max<uint64_t>(S->stats.max_inflight_bytes, S->inflight_bytes);
                S->stats.max_batch_msgs = 1;
            }
            S->stats.max_queue = std::max<uint64_t>(S->stats.max_queue, S->queue.size());
            publish_diagnostics(S);
        }
        inflight = !S->rinflight[0].empty() || !S->rinflight[1].empty();
        if (inflight && !S->rlive) {  // published work and no kernel: (re)launch
            const int rc = timed_cuda(S, [&] { return start_resident(S); });
            {
                SchedLock lk(S, kLockStats);
                S->stats.batches++;  // resident mode: kernel launches
            }
            if (rc == AES_OK) {
                S->rlive = true;
                S->rprogress_s = S->now();
            } else {
                fail_resident_inflight(S, rc);
            }
            worked = true;
        }
        end_phase(S, kPhaseLaunch, &ph);
        if (worked) {
            last_work = S->now();
        } else {
            // Nothing to do: keep polling for 200 us after the last work (a
            // condition-variable wake-up would add its latency to the next
            // request), then sleep until a submission.  Not while a kernel is
            // running or stopping: its end must be seen.
            const bool idle = S->queue.empty() && !inflight && !S->rlive;
            if (!idle_wait(S, idle && S->now() - last_work > 200e-6)) break;
        }
    }
    // Shutdown: everything has completed and the kernel has been stopped.
}

// Checks one request on the host (sizes, key, pointers); AES_OK or the error it is refused with.
static int check_request(aes_server* S, const aes_server_request& r, RangeCache* cache = nullptr) {
    if (r.key_index >= S->keys.size())
        return fail(AES_ERR_ARG, "request %llu: key_index %u >= %zu", (unsigned long long)r.id, r.key_index,
                    S->keys.size());
    if (r.decrypt > 1) return fail(AES_ERR_ARG, "request %llu: decrypt must be 0 or 1", (unsigned long long)r.id);
    if (r.nblocks > (UINT64_MAX >> 6)) return fail(AES_ERR_ARG, "request %llu: nblocks too large", (unsigned long long)r.id);
    if (request_bytes(r) > S->cfg.budget_bytes || r.nblocks > S->cfg.max_batch_blocks) {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        S->stats.rejected++;
        return fail(AES_ERR_BUDGET, "request %llu: %llu blocks exceed the server's budget or batch limit",
                    (unsigned long long)r.id, (unsigned long long)r.nblocks);
    }
    if (!S->dryrun && r.nblocks) {
        const size_t bytes = (size_t)r.nblocks * 16;
        int rc = check_device_range_cached(r.in, bytes, "request in", cache);
        if (!rc) rc = check_device_range_cached(r.out, bytes, "request out", cache);
        if (rc) return rc;
        const uintptr_t i0 = (uintptr_t)r.in, o0 = (uintptr_t)r.out;
        if (i0 != o0 && i0 < o0 + bytes && o0 < i0 + bytes) return fail(AES_ERR_ARG, "request in/out overlap partially");
    } else if (((uintptr_t)r.in | (uintptr_t)r.out) & 15u) {
        return fail(AES_ERR_ALIGN, "request %llu: pointers must be 16-byte aligned", (unsigned long long)r.id);
    }
    return AES_OK;
}

// Hands validated requests to the scheduler under one lock.
static void push_inbox(aes_server* S, const Pending* p, size_t n) {
    if (!n) return;
    S->submitted.fetch_add(n);
    {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        S->stats.submitted += n;
    }
    {
        std::lock_guard<std::mutex> lk(S->in_mu);
        const double t = S->now();
        S->inbox.insert(S->inbox.end(), p, p + n);
        S->inbox_n.store(S->inbox.size(), std::memory_order_release);
        const uint64_t held = (uint64_t)(1e9 * (S->now() - t));
        if (held > S->submit_hold_ns.load(std::memory_order_relaxed))
            S->submit_hold_ns.store(held, std::memory_order_relaxed);  // (submitters hold in_mu here)
    }
    S->in_cv.notify_one();
}

static int enqueue(aes_server* S, const aes_server_request& r, double arrival) {
    const int rc = check_request(S, r);
    if (rc) return rc;
    const Pending p{r, arrival};
    push_inbox(S, &p, 1);
    return AES_OK;
}

static void producer_main(aes_server* S) {
    pthread_setname_np(pthread_self(), "gbaes-replay");
    if (!S->dryrun) cudaSetDevice(S->device);  // (the stack registration and pool chunks use its context)
    const PinnedStackTop stack_top(!S->dryrun);
    if (S->cfg.flags & AES_SERVER_PIN_THREADS) S->producer_cpu = pin_thread(1);
    const double start = S->now();
    S->replay_start = start;
    // Lateness diagnostics: the thread's involuntary switches are read every
    // 16th hand-over and at any hand-over 20 us late or more.
    double cpu0 = 0;
    long inv_begin = 0, inv_prev = 0, flt_begin = 0;
    ThreadWatch::usage(&cpu0, &inv_begin, nullptr, &flt_begin);
    inv_prev = inv_begin;
    uint64_t handovers = 0;
    double late_max = 0, late_at = 0;
    long late_invol = 0;
    // Every request was checked when the replay was started (no driver call here).
    auto check = [&](size_t i) { return S->replay_rc[i]; };
    HotVec<Pending> due_now(HotAlloc<Pending>(&S->pool));
    const size_t n = S->replay_reqs.size();
    // Hands request r (already checked: rc) to the scheduler's batch, or
    // completes it at once with its error.
    auto take = [&](const aes_server_request& r, int rc) {
        const double t = start + r.arrival_s;
        if (rc == AES_OK) {
            due_now.push_back(Pending{r, t});
        } else {
            aes_server_completion c{r.id, rc, 0, t, t, S->now()};
            std::lock_guard<std::mutex> lk(S->out_mu);
            if (S->done.push(&c, 1) != 1) S->lost_completions.fetch_add(1);
        }
    };
    for (size_t i = 0; i < n;) {
        if (S->producer_stop.load()) break;
        // The next request is checked before its arrival time, so the driver
        // queries of the check are not part of its latency.
        const int rc_first = check(i);
        const double due = start + S->replay_reqs[i].arrival_s;
        for (;;) {  // wait for the scheduled arrival time: sleep, then yield, then spin for the last 50 us
            const double wait = due - S->now();
            if (wait <= 0) break;
            if (wait > 200e-6)
                std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
            else if (wait > 50e-6)
                std::this_thread::yield();
            if (S->producer_stop.load()) break;
        }
        if (S->producer_stop.load()) break;
        // Every request already due goes over in one hand-over (under load the
        // producer runs behind the schedule and several are due at once).
        due_now.clear();
        take(S->replay_reqs[i++], rc_first);
        const double now = S->now();
        for (; i < n && start + S->replay_reqs[i].arrival_s <= now; ++i)
            take(S->replay_reqs[i], check(i));
        push_inbox(S, due_now.data(), due_now.size());
        const double late = now - due;
        if (++handovers % 16 == 0 || late >= 20e-6) {
            double cpu;
            long inv;
            ThreadWatch::usage(&cpu, &inv);
            if (late > late_max) {
                late_max = late;
                late_at = due;
                late_invol = inv - inv_prev;
            }
            inv_prev = inv;
        }
    }
    {
        double cpu;
        long inv, flt;
        ThreadWatch::usage(&cpu, &inv, nullptr, &flt);
        std::lock_guard<std::mutex> lk(S->stats_mu);
        aes_server_diag& d = S->diag;
        d.producer_minflt += (uint64_t)(flt - flt_begin);
        if (late_max > 1e-9 * d.producer_late_max_ns) {
            d.producer_late_max_ns = (uint64_t)(1e9 * late_max);
            d.producer_late_at_ns = (uint64_t)(1e9 * late_at);
            d.producer_late_invol = (uint64_t)late_invol;
        }
        d.producer_invol += (uint64_t)(inv - inv_begin);
        d.producer_cpu = S->producer_cpu;
    }
    S->producer_running.store(false);
}

static void destroy_server(aes_server* S) {
    if (S->rctrl) {  // the scheduler has seen the kernel end; a safeguard before anything it reads is freed
        __atomic_store_n(&S->rctrl->stop, 1u, __ATOMIC_RELEASE);
        if (S->fake.joinable()) S->fake.join();
        if (S->rstream) cudaStreamSynchronize(S->rstream);
    }
    for (Slot& slot : S->slots) {
        if (slot.done) cudaEventDestroy(slot.done);
        if (slot.stream) cudaStreamDestroy(slot.stream);
        if (slot.dev_buf) cudaFree(slot.dev_buf);
        if (slot.host_buf) cudaFreeHost(slot.host_buf);
    }
    if (S->dev_keys) cudaFree(S->dev_keys);
    if (S->dryrun) {
        free(S->ring_mem);
    } else {
        if (S->ring_mem) cudaFreeHost(S->ring_mem);
        if (S->rargs.claim) cudaFree(S->rargs.claim);
        if (S->rargs.done) cudaFree(S->rargs.done);
        if (S->rargs.abandon) cudaFree(S->rargs.abandon);
        if (S->rargs.abandon_n) cudaFree(S->rargs.abandon_n);
        if (S->rargs.cq_next) cudaFree(S->rargs.cq_next);
        if (S->rstream) cudaStreamDestroy(S->rstream);
    }
    const bool locked = S->self_locked;
    S->~aes_server();
    free_host(S, locked);
}

static bool pow2(uint32_t x) { return x && !(x & (x - 1)); }

// Ring memory, counters and the kernel's stream for resident mode.
static int setup_resident(aes_server* S) {
    const aes_server_config& c = S->cfg;
    const uint32_t rt = c.ring_tiles, ri = c.ring_items;
    const uint32_t cq = 2 * ri;  // no more requests than this are in flight
    const size_t exit_off = sizeof(ResCtrl) + sizeof(ResTile) * 2 * (size_t)rt + sizeof(ResDone) * (size_t)cq;
    const size_t bytes = exit_off + sizeof(uint64_t) * kResidentMaxCtas;
    uint8_t* dev_view = nullptr;
    if (S->dryrun) {
        S->ring_mem = (uint8_t*)aligned_alloc(64, (bytes + 63) & ~(size_t)63);
        if (!S->ring_mem) return fail(AES_ERR_NOMEM, "out of host memory");
        dev_view = S->ring_mem;
        S->fake_claim.assign(2, 0);
        S->fake_done.assign(2 * (size_t)ri, 0);
    } else {
        int can_map = 0;
        cudaError_t e = cudaDeviceGetAttribute(&can_map, cudaDevAttrCanMapHostMemory, S->device);
        if (e == cudaSuccess && !can_map) return fail(AES_ERR_CUDA, "resident mode needs mapped page-locked memory");
        if (e == cudaSuccess) e = cudaHostAlloc(&S->ring_mem, bytes, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&dev_view, S->ring_mem, 0);
        if (e == cudaSuccess) e = cudaMalloc(&S->rargs.claim, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&S->rargs.done, 2 * (size_t)ri * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&S->rargs.abandon, 2 * (size_t)kAbandonCap * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&S->rargs.abandon_n, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&S->rargs.cq_next, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(S->rargs.cq_next, 0, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(S->rargs.abandon_n, 0, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(S->rargs.claim, 0, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(S->rargs.done, 0, 2 * (size_t)ri * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->rstream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? AES_ERR_NOMEM : AES_ERR_CUDA, "resident setup: %s",
                        cudaGetErrorString(e));
        }
    }
    memset(S->ring_mem, 0, bytes);
    S->rctrl = (ResCtrl*)S->ring_mem;
    S->rtiles = (ResTile*)(S->ring_mem + sizeof(ResCtrl));
    S->rcq = (ResDone*)(S->ring_mem + sizeof(ResCtrl) + sizeof(ResTile) * 2 * (size_t)rt);
    S->rargs.ctrl = (const ResCtrl*)dev_view;
    S->rargs.tiles = (const ResTile*)(dev_view + sizeof(ResCtrl));
    S->rargs.cq = (ResDone*)(dev_view + sizeof(ResCtrl) + sizeof(ResTile) * 2 * (size_t)rt);
    S->rexit = (uint64_t*)(S->ring_mem + exit_off);
    S->rargs.exit_gen = (uint64_t*)(dev_view + exit_off);
    S->rargs.cq_size = cq;
    S->rargs.cq_log2 = (uint32_t)__builtin_ctz(cq);
    S->rargs.keys = S->dev_keys;
    S->rargs.err = S->status;
    S->rargs.ring_tiles = rt;
    S->rargs.ring_items = ri;
    if (!S->dryrun) {
        DeviceInfo info;
        int rc = current_device_info(&info);
        if (rc) return rc;
        if ((uint32_t)info.sms > kResidentMaxCtas) return fail(AES_ERR_CUDA, "more SMs than resident CTAs supported");
        S->spread = (uint32_t)info.sms;
        S->rgrid = (uint32_t)info.sms;
    } else {
        S->spread = 8;
    }
    S->spread = std::min(S->spread, rt);  // a request never needs more ring than ring_tiles
    S->rargs.lifetime_ns = 1000000ull * c.resident_lifetime_ms;
    return AES_OK;
}

}  // namespace gbaes

extern "C" {

aes_server* aes_server_create(const aes_ctx* const* keys, size_t nkeys, const aes_server_config* config) {
    aes_server_config cfg;
    memset(&cfg, 0, sizeof cfg);
    if (config) cfg = *config;
    if (cfg.budget_bytes == 0) cfg.budget_bytes = (uint64_t)8 << 30;
    if (cfg.nstreams == 0) cfg.nstreams = 4;
    if (cfg.threads == 0) cfg.threads = 512;
    if (cfg.blocks_per_thread == 0) cfg.blocks_per_thread = (cfg.flags & AES_SERVER_RESIDENT) ? 2 : 1;
    if (cfg.max_batch_msgs == 0) cfg.max_batch_msgs = 4096;
    if (cfg.max_batch_blocks == 0) cfg.max_batch_blocks = (uint64_t)1 << 22;
    if (cfg.resident_idle_us == 0) cfg.resident_idle_us = 2000;
    if (cfg.resident_lifetime_ms == 0) cfg.resident_lifetime_ms = 10000;
    if (cfg.ring_tiles == 0) cfg.ring_tiles = 1u << 16;
    if (cfg.ring_items == 0) cfg.ring_items = 1u << 14;
    if (cfg.resident_restart_pct == 0) cfg.resident_restart_pct = 80;
    if (cfg.nstreams < 1 || cfg.nstreams > 64 || cfg.threads < 64 || cfg.threads > 1024 || cfg.threads % 32 ||
        (cfg.blocks_per_thread != 1 && cfg.blocks_per_thread != 2 && cfg.blocks_per_thread != 4) ||
        cfg.max_batch_msgs > (1u << 20) || (cfg.flags & ~(AES_SERVER_DRYRUN | AES_SERVER_RESIDENT | AES_SERVER_PIN_THREADS)) ||
        cfg.resident_restart_pct > 1000) {
        fail(AES_ERR_ARG, "invalid server configuration");
        return nullptr;
    }
    if ((cfg.flags & AES_SERVER_RESIDENT) && cfg.threads > (int)kResidentMaxThreads) {
        fail(AES_ERR_ARG, "resident mode: threads %d (at most %u compute threads per CTA)", cfg.threads,
             kResidentMaxThreads);
        return nullptr;
    }
    const uint64_t res_tile = (uint64_t)cfg.threads * (uint64_t)cfg.blocks_per_thread;
    if ((cfg.flags & AES_SERVER_RESIDENT) &&
        (!pow2(cfg.ring_tiles) || !pow2(cfg.ring_items) || cfg.ring_tiles > (1u << 24) || cfg.ring_items > (1u << 24) ||
         (cfg.max_batch_blocks + res_tile - 1) / res_tile > cfg.ring_tiles)) {
        fail(AES_ERR_ARG,
             "resident mode: ring_tiles and ring_items must be powers of two up to 2^24, and ring_tiles must hold "
             "the largest request (max_batch_blocks / (threads * blocks_per_thread) tiles)");
        return nullptr;
    }
    if (nkeys == 0 || !keys) {
        fail(AES_ERR_ARG, "a server needs at least one key");
        return nullptr;
    }
    for (size_t i = 0; i < nkeys; ++i)
        if (!keys[i] || keys[i]->magic != kCtxMagic) {
            fail(AES_ERR_ARG, "keys[%zu] is not a valid aes_ctx", i);
            return nullptr;
        }
    int host_device = -1;  // page-locked server data through this device's context (none in a dry run)
    if ((cfg.flags & AES_SERVER_DRYRUN) == 0 && cudaGetDevice(&host_device) != cudaSuccess) {
        cudaGetLastError();
        fail(AES_ERR_CUDA, "server setup: no current device");
        return nullptr;
    }
    bool locked = false;
    void* mem = alloc_host(sizeof(aes_server), host_device, &locked);
    if (!mem) {
        fail(AES_ERR_NOMEM, "out of host memory");
        return nullptr;
    }
    aes_server* S = new (mem) aes_server(host_device);
    S->self_locked = locked;
    S->cfg = cfg;
    S->dryrun = (cfg.flags & AES_SERVER_DRYRUN) != 0;
    S->resident = (cfg.flags & AES_SERVER_RESIDENT) != 0;
    S->tile_blocks = (uint32_t)res_tile;
    S->keys.assign(nkeys, aes_ctx{});
    for (size_t i = 0; i < nkeys; ++i) S->keys[i] = *keys[i];
    for (size_t i = 0; i < nkeys; ++i) S->key_ptrs.push_back(&S->keys[i]);
    if (!S->resident)
        for (int i = 0; i < cfg.nstreams; ++i) S->slots.emplace_back(&S->pool);
    const uint64_t tb = 32ull * cfg.blocks_per_thread;
    S->slot_cap = 256 + (((size_t)cfg.max_batch_msgs * sizeof(MsgDev) + 255) & ~(size_t)255) +
                  4 * (size_t)(cfg.max_batch_blocks / tb + 8) + 4;
    if (!S->dryrun) {
        cudaError_t e = cudaGetDevice(&S->device);
        std::vector<uint32_t> img(2 * nkeys * 64, 0u);
        for (size_t i = 0; i < nkeys; ++i) {
            memcpy(&img[(2 * i) * 64], keys[i]->enc_rk, 4 * 4 * (keys[i]->nr + 1));
            memcpy(&img[(2 * i + 1) * 64], keys[i]->dec_rk, 4 * 4 * (keys[i]->nr + 1));
        }
        if (e == cudaSuccess) e = cudaMalloc(&S->dev_keys, img.size() * 4);
        if (e == cudaSuccess) e = cudaMemcpy(S->dev_keys, img.data(), img.size() * 4, cudaMemcpyHostToDevice);
        for (Slot& slot : S->slots) {
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMalloc(&slot.dev_buf, S->slot_cap);
            if (e == cudaSuccess) e = cudaMallocHost(&slot.host_buf, S->slot_cap);
        }
        if (e != cudaSuccess || device_status_word(&S->status)) {
            fail(AES_ERR_CUDA, "server setup: %s", cudaGetErrorString(e));
            cudaGetLastError();
            destroy_server(S);
            return nullptr;
        }
    }
    if (S->resident && setup_resident(S) != AES_OK) {
        destroy_server(S);
        return nullptr;
    }
    S->done.set_device(S->dryrun ? -1 : S->device);
    S->done.reserve(kCompletionsAhead);  // (short of memory: completions then take pages as they come)
    S->stats.budget_bytes = cfg.budget_bytes;
    S->diag.sched_cpu = -1;
    S->diag.producer_cpu = -1;
    S->t0 = std::chrono::steady_clock::now();
    S->magic = kServerMagic;
    S->scheduler = std::thread(S->resident ? scheduler_resident : scheduler_main, S);
    return S;
}

static int check_server(aes_server* S) {
    if (!S || S->magic != kServerMagic) return fail(AES_ERR_ARG, "invalid aes_server");
    if (S->stop.load()) return fail(AES_ERR_STATE, "server is shutting down");
    return AES_OK;
}

int aes_server_submit(aes_server* S, const aes_server_request* r) {
    int rc = check_server(S);
    if (rc) return rc;
    if (!r) return fail(AES_ERR_ARG, "request is NULL");
    return enqueue(S, *r, S->now());
}

int aes_server_replay(aes_server* S, const aes_server_request* reqs, size_t n) {
    int rc = check_server(S);
    if (rc) return rc;
    if (n && !reqs) return fail(AES_ERR_ARG, "requests are NULL");
    if (S->producer_running.load() || S->producer.joinable())
        return fail(AES_ERR_STATE, "a replay is already running (join it first)");
    for (size_t i = 1; i < n; ++i)
        if (reqs[i].arrival_s < reqs[i - 1].arrival_s) return fail(AES_ERR_ARG, "arrival times must not decrease");
    S->replay_reqs.assign(reqs, reqs + n);
    // Checks every request now, not on the replay thread: its hand-overs then
    // make no driver call (a pointer query can wait behind the driver for tens of
    // milliseconds).  The caller keeps the buffers valid for the replay, so the
    // allocations found valid here stay valid, and a cache of them spares the
    // driver a query per request.
    S->replay_rc.resize(n);
    RangeCache cache;
    double check_max = 0, check_at = 0;
    for (size_t i = 0; i < n; ++i) {
        const double t = S->now();
        S->replay_rc[i] = check_request(S, reqs[i], &cache);
        if (S->now() - t > check_max) {
            check_max = S->now() - t;
            check_at = t;
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        if (check_max > 1e-9 * S->diag.producer_check_max_ns) {
            S->diag.producer_check_max_ns = (uint64_t)(1e9 * check_max);
            S->diag.producer_check_at_ns = (uint64_t)(1e9 * check_at);
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->out_mu);
        S->done.reserve(n + kCompletionsAhead);  // every completion of the replay lands on a page made now
    }
    clear_error();
    S->producer_stop.store(false);
    S->producer_running.store(true);
    S->producer = std::thread(producer_main, S);
    return AES_OK;
}

int aes_server_replay_join(aes_server* S, int stop_early) {
    if (!S || S->magic != kServerMagic) return fail(AES_ERR_ARG, "invalid aes_server");
    if (stop_early) S->producer_stop.store(true);
    if (S->producer.joinable()) S->producer.join();
    return AES_OK;
}

int aes_server_drain(aes_server* S, double timeout_s) {
    if (!S || S->magic != kServerMagic) return fail(AES_ERR_ARG, "invalid aes_server");
    const double until = S->now() + timeout_s;
    while (S->finished.load() < S->submitted.load() || S->producer_running.load()) {
        if (timeout_s >= 0 && S->now() > until) return fail(AES_ERR_STATE, "drain timed out");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return AES_OK;
}

int aes_server_poll(aes_server* S, aes_server_completion* out, size_t max) {
    if (!S || S->magic != kServerMagic) return fail(AES_ERR_ARG, "invalid aes_server");
    if (max && !out) return fail(AES_ERR_ARG, "out is NULL");
    if (max > 0x7FFFFFFF) max = 0x7FFFFFFF;  // (the count is returned as an int)
    std::lock_guard<std::mutex> lk(S->out_mu);
    return (int)S->done.pop(out, max);
}

int aes_server_get_stats(aes_server* S, aes_server_stats* out) {
    if (!S || S->magic != kServerMagic) return fail(AES_ERR_ARG, "invalid aes_server");
    if (!out) return fail(AES_ERR_ARG, "out is NULL");
    std::lock_guard<std::mutex> lk(S->stats_mu);
    *out = S->stats;
    out->lost_completions = S->lost_completions.load();
    return AES_OK;
}

int aes_server_get_diag(aes_server* S, aes_server_diag* out) {
    if (!S || S->magic != kServerMagic) return fail(AES_ERR_ARG, "invalid aes_server");
    if (!out) return fail(AES_ERR_ARG, "out is NULL");
    std::lock_guard<std::mutex> lk(S->stats_mu);
    *out = S->diag;
    return AES_OK;
}

int aes_server_cancel(aes_server* S, uint64_t id) {
    if (!S || S->magic != kServerMagic) return fail(AES_ERR_ARG, "invalid aes_server");
    {
        std::lock_guard<std::mutex> lk(S->in_mu);
        S->cancels.push_back(id);
        S->cancels_n.store(S->cancels.size(), std::memory_order_release);
    }
    S->in_cv.notify_one();
    return AES_OK;
}

int aes_server_inject_fault(aes_server* S, uint64_t batch_index) {
    if (!S || S->magic != kServerMagic) return fail(AES_ERR_ARG, "invalid aes_server");
    S->fault_batch.store(batch_index);
    return AES_OK;
}

void aes_server_destroy(aes_server* S) {
    if (!S || S->magic != kServerMagic) return;
    S->producer_stop.store(true);
    if (S->producer.joinable()) S->producer.join();
    S->stop.store(true);
    S->in_cv.notify_one();
    if (S->scheduler.joinable()) S->scheduler.join();
    S->magic = 0;
    destroy_server(S);
}

}  // extern "C"

// ------------------------------------------------------------------ routing

struct aes_router {
    uint32_t magic = 0;
    int policy = AES_ROUTE_LEAST_LOADED;
    std::vector<aes_server*> servers;
    std::mutex mu;       // the choice (and its round-robin cursor)
    size_t next = 0;     // round-robin start among equally loaded servers
    size_t poll_next = 0;
};

namespace gbaes {

constexpr uint32_t kRouterMagic = 0x524f5554u;  // "ROUT"

static bool valid_router(const aes_router* R) { return R && R->magic == kRouterMagic; }

// Device that holds the memory at p (device or managed memory), else -1.
static int device_of(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return -1;
    return a.device;
}

}  // namespace gbaes

extern "C" {

aes_router* aes_router_create(aes_server* const* servers, size_t n, int policy) {
    if (!servers || n == 0) {
        fail(AES_ERR_ARG, "a router needs at least one server");
        return nullptr;
    }
    if (policy != AES_ROUTE_LEAST_LOADED && policy != AES_ROUTE_BY_DEVICE) {
        fail(AES_ERR_ARG, "unknown routing policy %d", policy);
        return nullptr;
    }
    for (size_t i = 0; i < n; ++i) {
        if (!servers[i] || servers[i]->magic != kServerMagic) {
            fail(AES_ERR_ARG, "servers[%zu] is not a valid aes_server", i);
            return nullptr;
        }
        for (size_t j = 0; j < i; ++j)
            if (servers[j] == servers[i]) {
                fail(AES_ERR_ARG, "servers[%zu] repeats servers[%zu]", i, j);
                return nullptr;
            }
    }
    aes_router* R = new (std::nothrow) aes_router();
    if (!R) {
        fail(AES_ERR_NOMEM, "out of host memory");
        return nullptr;
    }
    R->policy = policy;
    R->servers.assign(servers, servers + n);
    R->magic = kRouterMagic;
    return R;
}

int aes_router_submit(aes_router* R, const aes_server_request* r) {
    if (!valid_router(R)) return fail(AES_ERR_ARG, "invalid aes_router");
    if (!r) return fail(AES_ERR_ARG, "request is NULL");
    const size_t n = R->servers.size();
    size_t pick = n;
    {
        std::lock_guard<std::mutex> lk(R->mu);
        // Candidates: the servers on the input's device (by-device policy),
        // else every server.
        int dev = -1;
        if (R->policy == AES_ROUTE_BY_DEVICE && r->nblocks) {
            dev = device_of(r->in);
            bool any = false;
            for (size_t i = 0; i < n && dev >= 0; ++i) any = any || (!R->servers[i]->dryrun && R->servers[i]->device == dev);
            if (!any) dev = -1;
        }
        // The least loaded candidate (unfinished requests), round robin among ties.
        uint64_t best = UINT64_MAX;
        for (size_t k = 0; k < n; ++k) {
            const size_t i = (R->next + k) % n;
            const aes_server* S = R->servers[i];
            if (dev >= 0 && (S->dryrun || S->device != dev)) continue;
            const uint64_t load = S->submitted.load() - S->finished.load();
            if (load < best) {
                best = load;
                pick = i;
            }
        }
        R->next = (pick + 1) % n;
    }
    const int rc = aes_server_submit(R->servers[pick], r);
    return rc == AES_OK ? (int)pick : rc;
}

int aes_router_poll(aes_router* R, aes_server_completion* out, size_t max) {
    if (!valid_router(R)) return fail(AES_ERR_ARG, "invalid aes_router");
    if (max && !out) return fail(AES_ERR_ARG, "out is NULL");
    if (max > 0x7FFFFFFF) max = 0x7FFFFFFF;
    size_t got = 0;
    const size_t n = R->servers.size();
    std::lock_guard<std::mutex> lk(R->mu);
    for (size_t k = 0; k < n && got < max; ++k) {  // start where the last poll stopped: no server starves
        const size_t i = (R->poll_next + k) % n;
        const int m = aes_server_poll(R->servers[i], out + got, max - got);
        if (m < 0) return m;
        got += (size_t)m;
    }
    R->poll_next = (R->poll_next + 1) % n;
    return (int)got;
}

int aes_router_drain(aes_router* R, double timeout_s) {
    if (!valid_router(R)) return fail(AES_ERR_ARG, "invalid aes_router");
    for (aes_server* S : R->servers) {
        const int rc = aes_server_drain(S, timeout_s);
        if (rc != AES_OK) return rc;
    }
    return AES_OK;
}

void aes_router_destroy(aes_router* R) {
    if (!valid_router(R)) return;
    R->magic = 0;
    delete R;
}

}  // extern "C"
