// Batched-launch data structures shared by the batch entry points (batch.cu)
// and the server (server.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gbaes_internal.h"

namespace gbaes {

struct MsgDev {  // 32 bytes, group order
    uint64_t blk_start;  // first block of the message in its group's block space
    uint64_t in_blk;     // in_off / 16
    uint64_t out_blk;    // out_off / 16
    uint32_t key_slot;   // schedule slot (2 * key_index + decrypt)
    uint32_t src;        // caller's message index
};

struct GroupDev {
    uint32_t tile_start, tile_end;  // tiles [tile_start, tile_end)
    uint32_t msg_start, msg_end;    // messages [msg_start, msg_end) in group order
    uint64_t blocks;                // blocks in the group
    int32_t nr;
    int32_t dir;  // 0 encrypt, 1 decrypt
};

constexpr int kGroups = 6;
constexpr int kSlotWords = 64;  // 60 used (Nr = 14), padded to 256 bytes

struct BatchArgs {
    const uint4* in;
    uint4* out;
    const MsgDev* msgs;
    const uint4* keys;  // kSlotWords / 4 uint4 per slot
    const uint32_t* tile_msg;
    unsigned* counter;
    int* status;
    uint32_t ntiles;
    uint32_t tile_blocks;
    GroupDev groups[kGroups];
};

struct HostPlan {
    std::vector<MsgDev> msgs;
    std::vector<uint32_t> tile_msg;
    std::vector<uint32_t> keys;  // 2 * nctx slots of kSlotWords words
    GroupDev groups[kGroups];
    uint32_t ntiles = 0;
    uint32_t tile_blocks = 0;
    uint64_t total_blocks = 0;
    uint64_t in_extent = 0;   // bytes from in_base the plan reads
    uint64_t out_extent = 0;  // bytes from out_base the plan writes
};

// Validates descriptors and lays out groups, tiles and (optionally) key slots.
int build_host_plan(const aes_msg_desc* d, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx, uint32_t tile_blocks,
                    bool with_keys, HostPlan* P);

// Launches the batched kernel (one CTA per SM at most; ntiles > 0).
int launch_batch_kernel(const BatchArgs& a, int threads, int bpt, cudaStream_t stream);

int device_status_word(int** p);  // ecb_table.cu

}  // namespace gbaes
