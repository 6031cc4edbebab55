// Request ring shared by the server's scheduler thread (server.cu) and the
// resident serving kernel (resident.cu).
//
// The host writes each admitted request as tile records into page-locked
// memory the GPU reads over the host link, then publishes them by advancing its
// direction's tile count (a release store).  CTAs of the resident kernel take
// tickets (tile indices) from a device-memory counter with an atomic add, also
// ahead of publication, and encipher a ticket's tile once it is published; they
// count finished blocks per request, and the CTA that finishes a request's last
// block appends (direction, request number) to a completion queue in
// page-locked memory, which the scheduler reads in order.  A CTA that leaves (stop
// word or lifetime) writes the tickets it still holds to the abandon list; once
// the kernel has ended, the host re-publishes the abandoned tiles that had been
// published meanwhile and moves the counters back to the first tile nobody took.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace gbaes {

// One tile: at most threads * blocks_per_thread consecutive blocks of one request.
struct ResTile {
    uint64_t in;           // device address of the tile's first input block
    uint64_t out;          // device address of its first output block
    uint64_t item_blocks;  // blocks of the whole request
    uint64_t seq;          // request number in its direction, from 1
    uint32_t nblocks;      // blocks in this tile (>= 1)
    uint32_t key_slot;     // schedule slot in the resident key table (2 * key index + direction)
    uint32_t item;         // request slot: index of its done counter
    uint32_t nr;           // rounds: 10, 12 or 14
};
static_assert(sizeof(ResTile) == 48, "tile records are three 16-byte words");

struct ResCtrl {
    uint64_t pub[2];  // tiles published per direction (only grows)
    uint32_t stop;    // non-zero: every CTA leaves at its next poll
    uint32_t pad[11];
};
static_assert(sizeof(ResCtrl) == 64, "one cache line");

constexpr uint32_t kAbandonCap = 1024;  // per direction (a CTA holds at most one ticket per direction)

// One completion: the i-th completion goes to entry i % cq_size as one word,
// written with a single release store:
//   lap << 40 | direction << 39 | (request number mod 2^39),
// where lap = (i / cq_size + 1) mod 2^24 tells the host a fresh entry from
// the one the previous lap left there (the host knows which lap it expects).
// At most cq_size requests are in flight, so an entry is always consumed
// before the next lap overwrites it, and 2^39 requests in flight can tell
// every request number from its low bits.
struct ResDone {
    uint64_t word;
};

constexpr uint64_t kCqSeqMask = (1ull << 39) - 1;

__host__ __device__ inline uint64_t cq_lap(uint64_t i, uint32_t cq_log2) { return ((i >> cq_log2) + 1) & 0xFFFFFFull; }

__host__ __device__ inline uint64_t cq_word(uint64_t i, uint32_t cq_log2, int dir, uint64_t seq) {
    return cq_lap(i, cq_log2) << 40 | (uint64_t)dir << 39 | (seq & kCqSeqMask);
}

struct ResArgs {
    const ResTile* tiles;           // [2][ring_tiles], device view of page-locked memory
    const ResCtrl* ctrl;            // device view of page-locked memory
    ResDone* cq;                    // [cq_size] completion queue, device view of page-locked memory
    unsigned long long* cq_next;    // device memory: completions written so far
    unsigned long long* claim;      // [2] device memory: next ticket (tile index) per direction
    unsigned long long* done;       // [2][ring_items] device memory: blocks finished per request slot
    unsigned long long* abandon;    // [2][kAbandonCap] device memory: tickets held by CTAs that left
    unsigned long long* abandon_n;  // [2] device memory: tickets written to the abandon list
    const uint4* keys;              // resident schedules, 256 bytes per slot
    int* err;                       // the library's device status word
    uint32_t ring_tiles;            // power of two
    uint32_t ring_items;            // power of two
    uint32_t cq_size;               // power of two, 2 * ring_items (requests in flight, both directions)
    uint32_t cq_log2;               // log2(cq_size)
    uint64_t lifetime_ns;           // a CTA leaves once this long has passed since its start
    uint64_t* exit_gen;             // [grid] device view of page-locked memory: gen once a CTA has left normally
    uint64_t gen;                   // this launch's number (from 1)
};

constexpr uint32_t kResidentMaxCtas = 1024;  // exit words in the ring memory (one per CTA)

// Compute threads per CTA of the resident kernel (at most; two control warps come on top).
constexpr uint32_t kResidentMaxThreads = 512;

// Launches the resident kernel: one CTA per SM, `threads` compute threads
// (64..kResidentMaxThreads, a multiple of 32) plus two control warps each, `bpt`
// (1, 2 or 4) blocks per compute thread per tile.
int launch_resident(const ResArgs& a, int threads, int bpt, cudaStream_t stream);

}  // namespace gbaes
