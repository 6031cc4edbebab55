// Resident serving kernel.
//
// The paper finds the per-operation overhead of each draw dominating small
// inputs and advises against small messages on the GPU (Section 3.1;
// Section 4).  The launch-per-batch server (server.cu) amortises launches over
// micro-batches but still pays a launch, a table upload and an event per
// batch.  In resident mode the kernel stays on the GPU instead: one CTA per SM
// holds the shared-memory tables of one direction and takes request tiles as
// the host publishes them into a ring in page-locked memory, which the GPU
// reads coherently over the host link (resident.h).  A tile is the CTA's unit
// of work: up to threads * BPT consecutive blocks of one request, thread i
// taking blocks i, i + threads, ... so every load and store is coalesced.
//
// Thread 0 takes tickets (tile indices) from the directions' device counters
// with atomic adds -- one always ready in its own direction, one in the other
// direction when that has published tiles nobody has taken -- polls the
// published-tile counts in page-locked memory, and copies a ticket's tile
// record into shared memory once the tile is published.  (Claiming by
// compare-and-swap instead serialised every claim behind one L2 atomic round
// trip per success: with 152 CTAs polling, ~38 failed swaps per claim.)  A CTA
// switches its tables to the other direction when its tile is there, so every
// live CTA serves every request.  Every thread fences its stores before the
// CTA's tile count goes into the request's done counter (an acquire-release
// add); the CTA that completes a request resets the counter and appends the
// request to the completion queue, the entry's tag last with a system-scope
// release.
//
// Every wait is bounded: a CTA leaves when the host sets the stop word or once
// lifetime_ns have passed since its start (both checked between tiles),
// writing the tickets it still holds to the abandon list.  The host stops the
// kernel (after it has stopped publishing) when it has been idle or is near
// its lifetime, and before relaunching re-publishes any abandoned tile that was
// published meanwhile and resets the ticket counters (resident.h).
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

// Thread 0: the next tile to encipher (true), or false when the CTA should
// leave.  One poll issues the loads of both published counts, the stop word
// and both ticket counters together (one host-link round trip).  The CTA
// always holds a ticket in its table direction `dir` (taken before the tile is
// published), and takes one in the other direction when that direction has
// published tiles nobody has taken.  It enciphers its own direction's tile
// when published, unless the other direction's held tile has been published
// for kMaxHoldNs (without that bound, a steady stream of own-direction work
// would starve it).  Before a tile's record is read, an acquire fence orders
// the read after the count that published it.  The CTA leaves on the stop
// word or its lifetime, unless a held ticket's tile has been published (it
// enciphers that first).
__device__ __forceinline__ bool next_tile(const ResArgs& a, int dir, uint64_t t_start, Tickets& tk, int* tdir,
                                          uint64_t* tile) {
    const int oth = dir ^ 1;
    for (;;) {
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
            return true;
        }
        if (stop || now - t_start > a.lifetime_ns) {
            load_pub(a, pub[0], pub[1]);  // fresh counts: a held tile published since the poll is enciphered first
            if ((tk.held[0] != kNoTicket && tk.held[0] < pub[0]) || (tk.held[1] != kNoTicket && tk.held[1] < pub[1]))
                continue;
            abandon_ticket(a, 0, tk.held[0]);
            abandon_ticket(a, 1, tk.held[1]);
            return false;
        }
        __nanosleep(200);
    }
}

template <int BPT>
__global__ void __launch_bounds__(1024, 1) resident_kernel(const ResArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t base = smem_base(smem_raw);
    const uint32_t A = table_base(base);
    const uint32_t end = (base + dynamic_smem_bytes()) & ~15u;
    // 64-byte control block (the claimed tile's record, a command and its
    // direction) and a 256-byte key slot: below the tables when the dynamic
    // window starts early enough, else above them.
    const uint32_t ctl = (A >= base + 320u) ? A - 320u : A + kDecBytes;
    const uint32_t kslot = ctl + 64u;
    if (A + kDecBytes > end || (ctl >= A && ctl + 320u > end)) {
        if (threadIdx.x == 0) atomicOr(a.err, 4);
        return;
    }
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t L0 = A | (lane << 2);
    const uint32_t L1 = L0 | 128u;
    int dir = (int)(blockIdx.x & 1u);
    fill_tables(A, dir != 0);
    const uint64_t t_start = globaltimer_ns();
    Tickets tk{{kNoTicket, kNoTicket}, {0, 0}};  // thread 0's tickets
    for (;;) {
        if (threadIdx.x == 0) {
            int tdir = dir;
            uint64_t tile = 0;
            uint32_t cmd = 1;
            if (next_tile(a, dir, t_start, tk, &tdir, &tile)) {
                const uint8_t* rec = (const uint8_t*)(a.tiles + (uint64_t)tdir * a.ring_tiles + (tile & (a.ring_tiles - 1)));
#pragma unroll
                for (int q = 0; q < 3; ++q) sts_v4(ctl + 16u * q, ld_volatile_v4(rec + 16 * q));
                cmd = 0;
            }
            sts(ctl + 48u, cmd);
            sts(ctl + 52u, (uint32_t)tdir);
        }
        __syncthreads();  // (also: every thread is done with the previous tile's tables, record and keys)
        if (lds(ctl + 48u)) break;
        const int tdir = (int)lds(ctl + 52u);
        if (tdir != dir) {
            fill_tables(A, tdir != 0);
            dir = tdir;
        }
        const uint4 r0 = lds_v4(ctl), r1 = lds_v4(ctl + 16u), r2 = lds_v4(ctl + 32u);
        const uint4* in = (const uint4*)(((uint64_t)r0.y << 32) | r0.x);
        uint4* out = (uint4*)(((uint64_t)r0.w << 32) | r0.z);
        const uint32_t n = r2.x, key_slot = r2.y, nr = r2.w;
        uint32_t s[BPT][4];
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const uint32_t i = threadIdx.x + (uint32_t)b * blockDim.x;
            const uint4 v = i < n ? ld_cg(in + i) : make_uint4(0, 0, 0, 0);
            s[b][0] = v.x;
            s[b][1] = v.y;
            s[b][2] = v.z;
            s[b][3] = v.w;
        }
        if (threadIdx.x <= nr) sts_v4(kslot + 16u * threadIdx.x, __ldg(a.keys + (uint64_t)key_slot * 16u + threadIdx.x));
        __syncthreads();  // the tables (after a swap) and the key slot are in place
        // Warps past the tile's last block skip the rounds, and every thread
        // runs only as many states as the tile fills (thread i has blocks i,
        // i + threads, ...): lookups on empty states would take shared-memory
        // cycles from the blocks that exist.  Small tiles thus cost what they
        // would with one block per thread, full ones amortise the tile's
        // fixed costs over BPT blocks per thread.
        if ((threadIdx.x & ~31u) < n) {
            const uint32_t states = (n + blockDim.x - 1) / blockDim.x;  // 1..BPT, the same in every thread
            if (states <= 1) {
                uint32_t(&s1)[1][4] = *reinterpret_cast<uint32_t(*)[1][4]>(&s[0]);
                if (dir)
                    cipher_rt<true, 1>(s1, SmemKeys{kslot}, (int)nr, L0, L1);
                else
                    cipher_rt<false, 1>(s1, SmemKeys{kslot}, (int)nr, L0, L1);
            } else if (BPT >= 4 && states <= 2) {
                uint32_t(&s2)[2][4] = *reinterpret_cast<uint32_t(*)[2][4]>(&s[0]);
                if (dir)
                    cipher_rt<true, 2>(s2, SmemKeys{kslot}, (int)nr, L0, L1);
                else
                    cipher_rt<false, 2>(s2, SmemKeys{kslot}, (int)nr, L0, L1);
            } else if (dir) {
                cipher_rt<true, BPT>(s, SmemKeys{kslot}, (int)nr, L0, L1);
            } else {
                cipher_rt<false, BPT>(s, SmemKeys{kslot}, (int)nr, L0, L1);
            }
        }
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const uint32_t i = threadIdx.x + (uint32_t)b * blockDim.x;
            if (i < n) out[i] = make_uint4(s[b][0], s[b][1], s[b][2], s[b][3]);
        }
        __threadfence();  // this thread's output before the tile is counted
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint64_t item_blocks = ((uint64_t)r1.y << 32) | r1.x;
            const uint64_t seq = ((uint64_t)r1.w << 32) | r1.z;
            const uint64_t slot = (uint64_t)dir * a.ring_items + r2.z;
            // A request of one tile is complete now: no count.  Otherwise the
            // count -- release: the CTA's outputs (fenced by every thread, then
            // the barrier) before it; acquire: the outputs of the tiles counted
            // before it.
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
                // The entry's tag is written last with a release store: it
                // orders the reset, the entry and every output this thread has
                // acquired (or its CTA wrote) before it; after it the host may
                // reuse the request's slot.
                const unsigned long long i = atomicAdd(a.cq_next, 1ull);
                ResDone* e = a.cq + (i & (a.cq_size - 1));
                asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(&e->what),
                             "l"(((uint64_t)dir << 63) | seq)
                             : "memory");
                st_release_sys(&e->tag, i + 1);
            }
        }
    }
}

using ResidentKernel = void (*)(const ResArgs);

int launch_resident(const ResArgs& a, int threads, int bpt, cudaStream_t stream) {
    ResidentKernel fn = bpt == 1 ? resident_kernel<1> : bpt == 2 ? resident_kernel<2> : bpt == 4 ? resident_kernel<4> : nullptr;
    if (!fn) return fail(AES_ERR_ARG, "blocks_per_thread %d: need 1, 2 or 4", bpt);
    if (threads < 64 || threads > 1024 || threads % 32) return fail(AES_ERR_ARG, "threads %d", threads);
    DeviceInfo info;
    int rc = current_device_info(&info);
    if (rc) return rc;
    rc = set_max_dynamic_smem((const void*)fn, info.smem_optin);
    if (rc) return rc;
    fn<<<info.sms, threads, info.smem_optin, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "resident kernel launch: %s", cudaGetErrorString(e));
    return AES_OK;
}

}  // namespace gbaes
