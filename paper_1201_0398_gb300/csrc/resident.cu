// Resident serving kernel.
//
// The paper finds the per-operation overhead of each draw dominating small
// inputs and advises against small messages on the GPU (Section 3.1;
// Section 4).  The launch-per-batch server (server.cu) amortises launches over
// micro-batches but still pays a launch, a table upload and an event per
// batch.  In resident mode the kernel stays on the GPU instead: one CTA per SM
// holds the shared-memory tables of one direction and takes request tiles as
// the host publishes them into a ring in page-locked memory, which the GPU
// reads coherently over the host link (resident.h).  A tile is the unit of
// work: up to C * BPT consecutive blocks of one request (C compute threads),
// thread i taking blocks i, i + C, ... so every load and store is coalesced.
//
// Each CTA is warp-specialised: C compute threads encipher, a producer lane
// takes tickets (tile indices) from the directions' device counters with
// atomic adds -- one always ready in its own direction, one in the other
// direction when that has published tiles nobody has taken -- polls the
// published-tile counts in page-locked memory and copies a ticket's tile
// record into shared memory once the tile is published, and a completer lane
// counts finished tiles into the request's done counter (an acquire-release
// add) and appends each finished request to the completion queue, the entry's
// tag last with a system-scope release.  (Claiming by compare-and-swap instead
// serialised every claim behind one L2 atomic round trip per success: with 152
// CTAs polling, ~38 failed swaps per claim.)  Two record slots let the
// producer stage tile i + 1 and the compute threads start loading its input
// while tile i is enciphered.  A CTA switches its tables to the other
// direction when its tile is there, so every live CTA serves every request.
//
// Every wait is bounded: a CTA leaves when the host sets the stop word or once
// lifetime_ns have passed since its start (both checked by the producer
// between tiles), writing the tickets it still holds to the abandon list.  The
// host stops the kernel (after it has stopped publishing) when it has been idle
// or is near its lifetime, and before relaunching re-publishes any abandoned
// tile that was published meanwhile and resets the ticket counters
// (resident.h).
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

#include "gbaes_internal.h"
#include "resident.h"
#include "rounds_rt.cuh"

namespace gbaes {

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint4 ld_volatile_v4(const void* p) {
    uint4 v;
    asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

// Input load cached in L2 only.  The kernel outlives many requests, whose
// buffers may be rewritten (by the caller, or by this kernel for in-place
// requests) while it runs, so neither the read-only path nor L1 may hold them.
__device__ __forceinline__ uint4 ld_cg(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void st_release_sys(uint64_t* p, uint64_t v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void sts_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ uint4 lds_v4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}

constexpr unsigned long long kNoTicket = ~0ull;

__device__ __forceinline__ void abandon_ticket(const ResArgs& a, int d, unsigned long long held) {
    if (held == kNoTicket) return;
    const unsigned long long i = atomicAdd(&a.abandon_n[d], 1ull);
    if (i < kAbandonCap)
        a.abandon[(uint64_t)d * kAbandonCap + i] = held;
    else
        atomicOr(a.err, 8);
}

__device__ __forceinline__ void load_pub(const ResArgs& a, uint64_t& p0, uint64_t& p1) {
    asm volatile("ld.relaxed.sys.global.v2.u64 {%0, %1}, [%2];" : "=l"(p0), "=l"(p1) : "l"(a.ctrl->pub) : "memory");
}

// The CTA's tickets (kept by thread 0 across tiles): held tile index per
// direction (kNoTicket if none) and when the CTA first saw that tile published
// (0: not yet).
struct Tickets {
    unsigned long long held[2];
    uint64_t ready[2];
};

// A published ticket of the other direction waits at most this long while the
// CTA keeps finding published tiles in its own direction.
constexpr uint64_t kMaxHoldNs = 20000;

// One poll of the producer lane (non-blocking): issues the loads of both
// published counts, the stop word and the other direction's ticket counter
// together (one host-link round trip).  The CTA always holds a ticket in
// direction `dir` -- the direction its tables will be in, i.e. that of the
// last tile it handed to its compute warps -- taken before the tile is
// published, and takes one in the other direction when that direction has
// published tiles nobody has taken.  It hands out its own direction's tile
// when published, unless the other direction's held tile has been published
// for kMaxHoldNs (without that bound, a steady stream of own-direction work
// would starve it).  Before a tile's record is read, an acquire fence orders
// the read after the count that published it.
// Returns kPollTile (*tdir, *tile set), kPollLeave (stop word or lifetime, and
// no held ticket's tile published: held tickets go to the abandon list) or
// kPollNothing.
constexpr int kPollNothing = 0, kPollTile = 1, kPollLeave = 2;

__device__ __forceinline__ int poll_tile(const ResArgs& a, int dir, uint64_t t_start, Tickets& tk, int* tdir,
                                         uint64_t* tile) {
    const int oth = dir ^ 1;
    const uint64_t now = globaltimer_ns() | 1u;  // (never 0: 0 marks "not seen published")
    uint64_t pub[2];
    load_pub(a, pub[0], pub[1]);
    const uint32_t stop = ld_volatile_u32(&a.ctrl->stop);
    const unsigned long long claim_oth = ld_volatile_u64(&a.claim[oth]);
    // Own / other direction views, by selects (no run-time index into a local array).
    const uint64_t pub_own = dir ? pub[1] : pub[0], pub_oth = dir ? pub[0] : pub[1];
    unsigned long long h_own = dir ? tk.held[1] : tk.held[0], h_oth = dir ? tk.held[0] : tk.held[1];
    uint64_t r_own = dir ? tk.ready[1] : tk.ready[0], r_oth = dir ? tk.ready[0] : tk.ready[1];
    if (h_own == kNoTicket) {
        h_own = atomicAdd(&a.claim[dir], 1ull);
        r_own = 0;
    }
    if (h_oth == kNoTicket && claim_oth < pub_oth) {
        h_oth = atomicAdd(&a.claim[oth], 1ull);
        r_oth = 0;
    }
    const bool own_ready = h_own < pub_own;
    const bool oth_ready = h_oth != kNoTicket && h_oth < pub_oth;
    if (own_ready && !r_own) r_own = now;
    if (oth_ready && !r_oth) r_oth = now;
    int got = -1;
    if (oth_ready && (!own_ready || now - r_oth > kMaxHoldNs))
        got = oth;
    else if (own_ready)
        got = dir;
    if (got == oth) {
        *tile = h_oth;
        h_oth = kNoTicket;
        r_oth = 0;
    } else if (got == dir) {
        *tile = h_own;
        h_own = kNoTicket;
        r_own = 0;
    }
    if (dir) {
        tk.held[1] = h_own;
        tk.held[0] = h_oth;
        tk.ready[1] = r_own;
        tk.ready[0] = r_oth;
    } else {
        tk.held[0] = h_own;
        tk.held[1] = h_oth;
        tk.ready[0] = r_own;
        tk.ready[1] = r_oth;
    }
    if (got >= 0) {
        asm volatile("fence.acq_rel.sys;" ::: "memory");
        *tdir = got;
        return kPollTile;
    }
    if (stop || now - t_start > a.lifetime_ns) {
        load_pub(a, pub[0], pub[1]);  // fresh counts: a held tile published since the poll is handed out first
        if ((tk.held[0] != kNoTicket && tk.held[0] < pub[0]) || (tk.held[1] != kNoTicket && tk.held[1] < pub[1]))
            return kPollNothing;
        abandon_ticket(a, 0, tk.held[0]);
        abandon_ticket(a, 1, tk.held[1]);
        tk.held[0] = tk.held[1] = kNoTicket;
        return kPollLeave;
    }
    return kPollNothing;
}

// ---------------------------------------------------------------- the kernel
//
// Warp-specialised: `C` compute threads (blockDim.x - 64) encipher tiles; two
// more warps, one lane each, do the rest so that none of it sits between two
// tiles of the compute warps.  The producer lane takes tickets and reads tile
// records; the completer lane counts finished tiles and completes requests.
// They share two slots in shared memory with the compute threads (double
// buffering): the producer fills slot i % 2 with tile i's record, its command
// (a tile, or leave) and direction while the compute warps work on tile i - 1,
// and the compute warps load tile i's input as soon as its slot is full --
// before enciphering tile i - 1 when the slot is already full then -- so the
// input's memory latency overlaps the previous tile's rounds.  Round keys come
// from the resident schedules through L1 (a warp-uniform 16-byte load per
// round, issued ahead of the round's lookups).  mbarriers in shared memory
// carry the hand-offs:
//   full[k]   1 arrival  (producer: slot k written)
//   empty[k]  C/32 arrivals (every compute warp: its outputs of slot k's tile stored)
//   free[k]   1 arrival  (completer: slot k's tile counted, the slot may be refilled)
//   sync      C/32 arrivals (the compute warps around a table fill)
// Every wait on them is bounded by the kernel's lifetime plus kGraceNs, after
// which the thread reports (status bit 16) and leaves; no hardware barrier is
// used after the start, so no thread can wait on one that has left.

constexpr uint32_t kSlotBytes = 64;                   // record (48 B), command, direction
constexpr uint32_t kCtlBytes = 2 * kSlotBytes + 64;   // two slots + seven mbarriers
constexpr uint32_t kCtlWarps = 2;                     // producer and completer
constexpr uint64_t kGraceNs = 1000000000ull;

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(addr)
                 : "memory");
}

// Non-blocking: has the phase of this parity completed?
__device__ __forceinline__ bool mbar_test(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of this parity, until `deadline` (globaltimer ns): false if it passed.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, uint64_t deadline) {
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
        if (globaltimer_ns() > deadline) return false;
    }
}

// Barrier of the C compute threads alone, on an mbarrier of one arrival per
// compute warp (so that it too gives up at the deadline instead of waiting on a
// thread that has left); phase: this thread's parity for its next use.
__device__ __forceinline__ bool compute_sync(uint32_t mb, uint32_t& phase, uint64_t deadline) {
    __syncwarp();  // (orders the warp's accesses before its arrival)
    if ((threadIdx.x & 31u) == 0) mbar_arrive(mb);
    const bool ok = mbar_wait(mb, phase, deadline);
    phase ^= 1u;
    return ok;
}

struct CtlBarriers {
    uint32_t full, empty, free_, sync;  // addresses of full[0], empty[0], free[0] (slot 1: + 8) and sync
};

// The completer counts a finished tile (slot sl) and, if it completes its
// request, appends the request to the completion queue.
__device__ __forceinline__ void account_tile(const ResArgs& a, uint32_t sl) {
    const uint4 r1 = lds_v4(sl + 16u), r2 = lds_v4(sl + 32u);
    const uint32_t dir = lds(sl + 52u);
    const uint32_t n = r2.x;
    const uint64_t item_blocks = ((uint64_t)r1.y << 32) | r1.x;
    const uint64_t seq = ((uint64_t)r1.w << 32) | r1.z;
    const uint64_t slot = (uint64_t)dir * a.ring_items + r2.z;
    // The compute warps stored the tile's outputs before their releasing
    // arrivals on the slot's empty barrier, which this lane has acquired: the
    // releases below (the count's, the completion's) order those outputs
    // before them at their own scope.
    // A request of one tile is complete now: no count.  Otherwise the count --
    // release: the tile's outputs before it; acquire: the outputs of the tiles
    // counted before it.
    bool last = n == item_blocks;
    if (!last) {
        unsigned long long before;
        asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
                     : "=l"(before)
                     : "l"(a.done + slot), "l"((unsigned long long)n)
                     : "memory");
        last = before + n == item_blocks;  // every other tile was counted before
        // No other CTA touches the counter now: reset it for the slot's next request.
        if (last) asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(a.done + slot), "l"(0ull) : "memory");
    }
    if (last) {
        // One release store writes the entry: it orders the reset and every
        // output this lane has acquired before it; after it the host may reuse
        // the request's slot.
        const unsigned long long i = atomicAdd(a.cq_next, 1ull);
        st_release_sys(&a.cq[i & (a.cq_size - 1)].word, cq_word(i, a.cq_log2, (int)dir, seq));
    }
}

// The producer lane: fills slot i % 2 once the completer has freed it from
// tile i - 2, with the next tile the ticket logic gives, or with "leave".
__device__ __forceinline__ void producer_lane(const ResArgs& a, uint32_t ctl, const CtlBarriers& mb, int dir,
                                              uint64_t t_start, uint64_t deadline) {
    Tickets tk{{kNoTicket, kNoTicket}, {0, 0}};
    for (uint32_t i = 0;; ++i) {
        const uint32_t k = i & 1u, sl = ctl + kSlotBytes * k;
        if (i >= 2 && !mbar_wait(mb.free_ + 8u * k, ((i - 2) >> 1) & 1u, deadline)) {
            atomicOr(a.err, 16);
            abandon_ticket(a, 0, tk.held[0]);
            abandon_ticket(a, 1, tk.held[1]);
            return;
        }
        for (;;) {
            int tdir = dir;
            uint64_t tile = 0;
            const int r = poll_tile(a, dir, t_start, tk, &tdir, &tile);
            if (r == kPollTile) {
                const uint8_t* rec =
                    (const uint8_t*)(a.tiles + (uint64_t)tdir * a.ring_tiles + (tile & (a.ring_tiles - 1)));
                const uint4 q0 = ld_volatile_v4(rec), q1 = ld_volatile_v4(rec + 16), q2 = ld_volatile_v4(rec + 32);
                sts_v4(sl, q0);
                sts_v4(sl + 16u, q1);
                sts_v4(sl + 32u, q2);
                sts(sl + 48u, 0u);
                sts(sl + 52u, (uint32_t)tdir);
                mbar_arrive(mb.full + 8u * k);
                dir = tdir;
                break;
            }
            if (r == kPollLeave) {  // (poll_tile gave up the held tickets)
                sts(sl + 48u, 1u);
                mbar_arrive(mb.full + 8u * k);
                return;
            }
            __nanosleep(100);
        }
    }
}

// The completer lane: in order, waits for tile i's slot to be full (leaves on
// "leave") and for the compute threads to have stored its outputs, counts it,
// and frees the slot.
__device__ __forceinline__ void completer_lane(const ResArgs& a, uint32_t ctl, const CtlBarriers& mb,
                                               uint64_t deadline) {
    for (uint32_t i = 0;; ++i) {
        const uint32_t k = i & 1u, par = (i >> 1) & 1u, sl = ctl + kSlotBytes * k;
        if (!mbar_wait(mb.full + 8u * k, par, deadline)) break;
        if (lds(sl + 48u)) {
            // Every tile this CTA was handed is counted: mark its exit in page-locked
            // memory, so that the host sees the kernel end without asking the driver.
            st_release_sys(a.exit_gen + blockIdx.x, a.gen);
            return;
        }
        if (!mbar_wait(mb.empty + 8u * k, par, deadline)) break;
        account_tile(a, sl);
        mbar_arrive(mb.free_ + 8u * k);
    }
    atomicOr(a.err, 16);
}

// Issues the loads of slot sl's tile: thread tid takes blocks tid, tid + C, ...
template <int BPT>
__device__ __forceinline__ void load_states(uint32_t sl, uint32_t tid, uint32_t C, uint32_t (&s)[BPT][4]) {
    const uint4 r0 = lds_v4(sl);
    const uint32_t n = lds(sl + 32u);
    const uint4* in = (const uint4*)(((uint64_t)r0.y << 32) | r0.x);
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const uint32_t i = tid + (uint32_t)b * C;
        const uint4 v = i < n ? ld_cg(in + i) : make_uint4(0, 0, 0, 0);
        s[b][0] = v.x;
        s[b][1] = v.y;
        s[b][2] = v.z;
        s[b][3] = v.w;
    }
}

template <int BPT>
__global__ void __launch_bounds__(kResidentMaxThreads + 32 * kCtlWarps, 1) resident_kernel(const ResArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t base = smem_base(smem_raw);
    const uint32_t A = table_base(base);
    const uint32_t end = (base + dynamic_smem_bytes()) & ~15u;
    // The control block (two slots and seven mbarriers): below the tables when
    // the dynamic window starts early enough, else above them.
    const uint32_t ctl = (A >= base + kCtlBytes) ? A - kCtlBytes : A + kDecBytes;
    if (A + kDecBytes > end || (ctl >= A && ctl + kCtlBytes > end)) {
        if (threadIdx.x == 0) atomicOr(a.err, 4);
        return;
    }
    const uint32_t C = blockDim.x - 32u * kCtlWarps;  // compute threads; then the producer and completer warps
    CtlBarriers mb;
    mb.full = ctl + 2 * kSlotBytes;
    mb.empty = mb.full + 16u;
    mb.free_ = mb.full + 32u;
    mb.sync = mb.full + 48u;
    const uint32_t full = mb.full, empty = mb.empty, sync_mb = mb.sync;
    if (threadIdx.x == 0) {
        mbar_init(full, 1);
        mbar_init(full + 8u, 1);
        mbar_init(empty, C / 32u);
        mbar_init(empty + 8u, C / 32u);
        mbar_init(mb.free_, 1);
        mbar_init(mb.free_ + 8u, 1);
        mbar_init(sync_mb, C / 32u);
    }
    __syncthreads();
    const uint64_t t_start = globaltimer_ns();
    const uint64_t deadline = t_start + a.lifetime_ns + kGraceNs;
    int dir = (int)(blockIdx.x & 1u);
    if (threadIdx.x >= C) {  // one lane of each control warp works, the others leave now
        if (threadIdx.x == C)
            producer_lane(a, ctl, mb, dir, t_start, deadline);
        else if (threadIdx.x == C + 32u)
            completer_lane(a, ctl, mb, deadline);
        return;
    }
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31u;
    const uint32_t L0 = A | (lane << 2);
    const uint32_t L1 = L0 | 128u;
    uint32_t sync_phase = 0;
    fill_tables_n(A, dir != 0, tid, C);
    if (!compute_sync(sync_mb, sync_phase, deadline)) {
        atomicOr(a.err, 16);
        return;
    }
    uint32_t s[BPT][4], sn[BPT][4];
    if (!mbar_wait(full, 0, deadline)) {
        atomicOr(a.err, 16);
        return;
    }
    if (lds(ctl + 48u)) return;  // leave before any tile
    load_states<BPT>(ctl, tid, C, s);
    for (uint32_t i = 0;; ++i) {
        const uint32_t sl = ctl + kSlotBytes * (i & 1u), sn_l = ctl + kSlotBytes * ((i + 1) & 1u);
        const uint32_t full_n = full + 8u * ((i + 1) & 1u), par_n = ((i + 1) >> 1) & 1u;
        // Tile i + 1 handed out already: issue its loads before tile i's rounds.
        const bool early = mbar_test(full_n, par_n);
        const bool leave_early = early && lds(sn_l + 48u) != 0;
        if (early && !leave_early) load_states<BPT>(sn_l, tid, C, sn);
        const uint4 r0 = lds_v4(sl), r2 = lds_v4(sl + 32u);
        const int tdir = (int)lds(sl + 52u);
        if (tdir != dir) {  // swap the tables (every compute thread is done with the old ones first)
            bool ok = compute_sync(sync_mb, sync_phase, deadline);
            if (ok) fill_tables_n(A, tdir != 0, tid, C);
            if (!ok || !compute_sync(sync_mb, sync_phase, deadline)) {
                atomicOr(a.err, 16);
                return;
            }
            dir = tdir;
        }
        uint4* out = (uint4*)(((uint64_t)r0.w << 32) | r0.z);
        const uint32_t n = r2.x, nr = r2.w;
        const OneGlobalKey keys{a.keys + (uint64_t)r2.y * 16u};
        // Warps past the tile's last block skip the rounds, and every thread
        // runs only as many states as the tile fills (thread i has blocks i,
        // i + C, ...): lookups on empty states would take shared-memory
        // cycles from the blocks that exist.  Small tiles thus cost what they
        // would with one block per thread, full ones amortise the tile's
        // fixed costs over BPT blocks per thread.
        if ((tid & ~31u) < n) {
            const uint32_t states = (n + C - 1) / C;  // 1..BPT, the same in every thread
            if (states <= 1) {
                uint32_t(&s1)[1][4] = *reinterpret_cast<uint32_t(*)[1][4]>(&s[0]);
                if (dir)
                    cipher_rt<true, 1>(s1, keys, (int)nr, L0, L1);
                else
                    cipher_rt<false, 1>(s1, keys, (int)nr, L0, L1);
            } else if (BPT >= 4 && states <= 2) {
                uint32_t(&s2)[2][4] = *reinterpret_cast<uint32_t(*)[2][4]>(&s[0]);
                if (dir)
                    cipher_rt<true, 2>(s2, keys, (int)nr, L0, L1);
                else
                    cipher_rt<false, 2>(s2, keys, (int)nr, L0, L1);
            } else if (dir) {
                cipher_rt<true, BPT>(s, keys, (int)nr, L0, L1);
            } else {
                cipher_rt<false, BPT>(s, keys, (int)nr, L0, L1);
            }
        }
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const uint32_t j = tid + (uint32_t)b * C;
            if (j < n) out[j] = make_uint4(s[b][0], s[b][1], s[b][2], s[b][3]);
        }
        __syncwarp();  // the warp's outputs before its arrival, which releases them to the completer
        if (lane == 0) mbar_arrive(empty + 8u * (i & 1u));
        if (leave_early) return;
        if (!early) {
            if (!mbar_wait(full_n, par_n, deadline)) {
                atomicOr(a.err, 16);
                return;
            }
            if (lds(sn_l + 48u)) return;
            load_states<BPT>(sn_l, tid, C, sn);
        }
#pragma unroll
        for (int b = 0; b < BPT; ++b)
#pragma unroll
            for (int w = 0; w < 4; ++w) s[b][w] = sn[b][w];
    }
}

using ResidentKernel = void (*)(const ResArgs);

int launch_resident(const ResArgs& a, int threads, int bpt, cudaStream_t stream) {
    ResidentKernel fn = bpt == 1 ? resident_kernel<1> : bpt == 2 ? resident_kernel<2> : bpt == 4 ? resident_kernel<4> : nullptr;
    if (!fn) return fail(AES_ERR_ARG, "blocks_per_thread %d: need 1, 2 or 4", bpt);
    if (threads < 64 || threads > (int)kResidentMaxThreads || threads % 32)
        return fail(AES_ERR_ARG, "resident kernel: threads %d (need a multiple of 32 in [64, %u])", threads,
                    kResidentMaxThreads);
    DeviceInfo info;
    int rc = current_device_info(&info);
    if (rc) return rc;
    rc = set_max_dynamic_smem((const void*)fn, info.smem_optin);
    if (rc) return rc;
    fn<<<info.sms, threads + 32 * kCtlWarps, info.smem_optin, stream>>>(a);  // + the producer and completer warps
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "resident kernel launch: %s", cudaGetErrorString(e));
    return AES_OK;
}

}  // namespace gbaes
