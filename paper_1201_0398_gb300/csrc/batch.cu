// Batched multi-key AES-ECB: many messages, each with its own key, key size and
// direction, in one persistent launch.
//
// The paper's draw-per-buffer design pays a per-operation overhead that
// dominates small inputs (Section 3.1; its conclusion advises against small
// messages).  Here thousands of messages share one launch:
//
//  * Host plan (batch_plan.h).  Messages are grouped by (direction, key size)
//    -- encryption groups first -- and each group's blocks are numbered
//    contiguously.  The flattened block space is cut into tiles; for every tile
//    the plan records the first message it touches.  Each (key, direction)
//    gets a slot holding its 4*(Nr+1)-word schedule.  Everything sits in one
//    device buffer, uploaded once per plan.
//  * Kernel.  One CTA per SM holds the shared-memory tables of aes_rounds.cuh.
//    Each *warp* starts on a fixed tile, then takes tiles from its
//    direction's atomic counter on its own, so the dependent loads at the
//    start of one warp's tile overlap the other warps' lookups; the CTA meets
//    at a barrier only to swap its tables from the encryption to the
//    decryption set, once.  A block finds its message
//    by binary search over the tile's message range (none when the tile lies
//    in one message); a warp whose tile lies in one message stages that
//    message's schedule in its shared-memory key slot, other tiles read keys
//    from global memory through L1.  The round count is a run-time loop bound,
//    so one compact body per direction serves all key sizes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "aes_rounds.cuh"
#include "batch_plan.h"
#include "rounds_rt.cuh"

namespace gbaes {

constexpr uint32_t kPlanTileMax = 512;  // largest tile of a batch plan, in blocks

// A tile inside one message m (the common case): blocks [tb0, tb0 + n) of the
// group's block space map to consecutive blocks of m, processed 32*BPT at a
// time (lane l, slot b -> block it + 32b + l, so every load and store
// instruction of the warp covers 512 contiguous bytes).  The descriptor is
// read once and m's schedule is staged in the warp's shared-memory key slot:
// one parallel load instead of a dependent global load per round, issued once
// the first data loads are in flight so that the two overlap.  Lanes past the
// end compute on zeros and store nothing, so the warp stays converged.
template <bool DEC, int BPT>
__device__ __forceinline__ void single_message_tile(const BatchArgs& a, const GroupDev& G, uint32_t m, uint64_t tb0,
                                                    uint32_t lane, uint32_t L0, uint32_t L1, uint32_t kslot) {
    const uint4* mp = (const uint4*)(a.msgs + m);
    const uint4 q0 = __ldg(mp);
    const uint4 q1 = __ldg(mp + 1);
    const uint64_t off = tb0 - (((uint64_t)q0.y << 32) | q0.x);  // tb0 - blk_start
    const uint4* in = a.in + ((((uint64_t)q0.w << 32) | q0.z) + off);
    uint4* out = a.out + ((((uint64_t)q1.y << 32) | q1.x) + off);
    const uint64_t left = G.blocks - tb0;
    const uint32_t n = left < a.tile_blocks ? (uint32_t)left : a.tile_blocks;
    for (uint32_t it = 0; it < n; it += 32u * BPT) {
        uint32_t s[BPT][4];
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const uint32_t i = it + 32u * b + lane;
            const uint4 v = i < n ? ld_stream(in + i) : make_uint4(0, 0, 0, 0);
            s[b][0] = v.x;
            s[b][1] = v.y;
            s[b][2] = v.z;
            s[b][3] = v.w;
        }
        if (it == 0) {  // (every lane has left the previous tile: the warp met at the tile-index shuffle)
            if (lane < (uint32_t)G.nr + 1u) {
                const uint4 k = __ldg(a.keys + (uint64_t)q1.z * (kSlotWords / 4) + lane);
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(kslot + 16u * lane), "r"(k.x),
                             "r"(k.y), "r"(k.z), "r"(k.w)
                             : "memory");
            }
            __syncwarp();
        }
        cipher_rt<DEC, BPT>(s, SmemKeys{kslot}, G.nr, L0, L1);
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const uint32_t i = it + 32u * b + lane;
            if (i < n) __stcs(out + i, make_uint4(s[b][0], s[b][1], s[b][2], s[b][3]));
        }
    }
}

// A tile that crosses message boundaries (messages m_lo..m_hi, m_lo < m_hi):
// each block finds its message by binary search over that range and reads its
// round keys from global memory through L1.  The states of one thread may
// belong to different messages: each carries its own key pointer, so the
// warp runs one interleaved cipher over all of them (no divergent per-block
// ciphers at a message boundary).
template <bool DEC, int BPT>
__device__ __forceinline__ void mixed_tile(const BatchArgs& a, const GroupDev& G, uint32_t m_lo, uint32_t m_hi,
                                           uint64_t tb0, uint32_t lane, uint32_t L0, uint32_t L1) {
    for (uint32_t it = 0; it < a.tile_blocks; it += 32u * BPT) {
        uint32_t s[BPT][4];
        uint64_t oidx[BPT];
        const uint4* kp[BPT];
        bool ok[BPT];
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const uint64_t gb = tb0 + it + 32u * b + lane;
            ok[b] = gb < G.blocks && it + 32u * b + lane < a.tile_blocks;
            uint4 v = make_uint4(0, 0, 0, 0);
            kp[b] = nullptr;
            oidx[b] = 0;
            if (ok[b]) {
                uint32_t lo = m_lo, hi = m_hi;  // largest m in [m_lo, m_hi] with blk_start[m] <= gb
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (__ldg((const unsigned long long*)(a.msgs + mid)) <= gb)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                const uint4* mp = (const uint4*)(a.msgs + lo);
                const uint4 r0 = __ldg(mp);
                const uint4 r1 = __ldg(mp + 1);
                const uint64_t blk_start = ((uint64_t)r0.y << 32) | r0.x;
                const uint64_t in_blk = ((uint64_t)r0.w << 32) | r0.z;
                const uint64_t out_blk = ((uint64_t)r1.y << 32) | r1.x;
                const uint64_t off = gb - blk_start;
                v = ld_stream(a.in + in_blk + off);
                oidx[b] = out_blk + off;
                kp[b] = a.keys + (uint64_t)r1.z * (kSlotWords / 4);
            }
            s[b][0] = v.x;
            s[b][1] = v.y;
            s[b][2] = v.z;
            s[b][3] = v.w;
        }
        if (!ok[0]) return;  // blocks only increase: nothing left in this tile for this lane
#pragma unroll
        for (int b = 1; b < BPT; ++b)
            if (!ok[b]) kp[b] = kp[0];  // (past the end: computes on zeros with a valid key, stores nothing)
        cipher_rt<DEC, BPT>(s, StateKeys<BPT>{kp}, G.nr, L0, L1);
#pragma unroll
        for (int b = 0; b < BPT; ++b)
            if (ok[b]) __stcs(a.out + oidx[b], make_uint4(s[b][0], s[b][1], s[b][2], s[b][3]));
    }
}

// One warp's tile t of group G: tile_blocks consecutive blocks of the group's
// block space (fewer in the group's last tile).
template <bool DEC, int BPT>
__device__ __forceinline__ void batch_warp_tile(const BatchArgs& a, const GroupDev& G, uint32_t t, uint32_t lane,
                                                uint32_t L0, uint32_t L1, uint32_t kslot) {
    const uint64_t tb0 = (uint64_t)(t - G.tile_start) * a.tile_blocks;
    const uint32_t m_lo = a.tile_msg[t];
    const uint32_t m_hi = (t + 1 < G.tile_end) ? a.tile_msg[t + 1] : G.msg_end - 1;
    if (m_lo == m_hi)
        single_message_tile<DEC, BPT>(a, G, m_lo, tb0, lane, L0, L1, kslot);
    else
        mixed_tile<DEC, BPT>(a, G, m_lo, m_hi, tb0, lane, L0, L1);
}

// Group table staged in shared memory (read with a runtime index per tile).
__device__ __forceinline__ GroupDev load_group(uint32_t gaddr, int g) {
    GroupDev G;
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = lds(gaddr + 32u * g + 4u * i);
    G.tile_start = w[0];
    G.tile_end = w[1];
    G.msg_start = w[2];
    G.msg_end = w[3];
    G.blocks = ((uint64_t)w[5] << 32) | w[4];
    G.nr = (int32_t)w[6];
    G.dir = (int32_t)w[7];
    return G;
}

// Tiles [0, E) are encryption tiles (groups 0-2), [E, ntiles) decryption
// tiles, with E = tile_end of group 2.  Every warp starts on a fixed tile,
// then takes tiles from the direction's own counter until it runs dry,
// independently of the other warps, so their global-memory latencies overlap.
// The CTA meets at a barrier only to swap its shared-memory tables from the
// encryption to the decryption set, once.
template <int BPT>
__global__ void __launch_bounds__(BPT == 8 ? 512 : 1024, 1) batch_kernel(const BatchArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t base = smem_base(smem_raw);
    const uint32_t A = table_base(base);
    const uint32_t gaddr = ((base + dynamic_smem_bytes()) & ~15u) - 32u * kGroups;  // group table
    // 256 B of key slot per warp: below the 64 KiB-aligned tables when the
    // dynamic window starts early enough, else above them.
    const uint32_t kslots = (A >= base + 256u * 32u) ? A - 256u * 32u : A + kDecBytes;
    if (A + kDecBytes > gaddr || (kslots >= A && kslots + 256u * 32u > gaddr)) {
        if (threadIdx.x == 0) atomicOr(a.status, 2);
        return;
    }
#pragma unroll
    for (int i = 0; i < kGroups; ++i) {
        if (threadIdx.x == (unsigned)i) {
            const GroupDev& G = a.groups[i];
            const uint32_t w[8] = {G.tile_start, G.tile_end, G.msg_start, G.msg_end, (uint32_t)G.blocks,
                                   (uint32_t)(G.blocks >> 32), (uint32_t)G.nr, (uint32_t)G.dir};
#pragma unroll
            for (int k = 0; k < 8; ++k) sts(gaddr + 32u * i + 4u * k, w[k]);
        }
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t L0 = A | (lane << 2);
    const uint32_t L1 = L0 | 128u;
    const uint32_t kslot = kslots + 256u * (threadIdx.x >> 5);
    const uint32_t enc_end = lds(gaddr + 32u * 2 + 4u);  // tile_end of group 2
    int cur_dir = -1;
    for (int dir = 0; dir < 2; ++dir) {
        const uint32_t t_begin = dir ? enc_end : 0u;
        const uint32_t t_end = dir ? a.ntiles : enc_end;
        if (t_begin >= t_end) continue;  // same for the whole CTA
        if (dir != cur_dir) {
            __syncthreads();  // every warp has left the other direction's tiles
            fill_tables(A, dir != 0);
            __syncthreads();
            cur_dir = dir;
        }
        // Every warp's first tile is fixed (interleaved over the CTAs, so a
        // small batch spreads over the SMs); later ones come from the
        // direction's counter, offset by the number of fixed tiles.
        const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
        uint32_t t = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
        while (t < t_end - t_begin) {
            uint32_t nxt = 0;
            if (lane == 0) nxt = atomicAdd(a.counter + dir, 1u) + nwarps;  // consumed after this tile
            t += t_begin;
            int g = 0;
            while (g < kGroups - 1 && t >= lds(gaddr + 32u * g + 4u)) ++g;  // tile_end of group g
            const GroupDev G = load_group(gaddr, g);
            if (dir)
                batch_warp_tile<true, BPT>(a, G, t, lane, L0, L1, kslot);
            else
                batch_warp_tile<false, BPT>(a, G, t, lane, L0, L1, kslot);
            t = __shfl_sync(0xffffffffu, nxt, 0);
        }
    }
}

// ------------------------------------------------------------------ host plan

static int group_of(int nr, int dir) { return dir * 3 + (nr == 10 ? 0 : nr == 12 ? 1 : 2); }

// Validates the descriptors and lays out groups, tiles and key slots.
int build_host_plan(const aes_msg_desc* d, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx,
                           uint32_t tile_blocks, bool with_keys, HostPlan* P) {
    if (nmsg && !d) return fail(AES_ERR_ARG, "message descriptors are NULL");
    if (nctx && !ctxs) return fail(AES_ERR_ARG, "key contexts are NULL");
    if (nmsg > 0xFFFFFFF0u) return fail(AES_ERR_ARG, "too many messages (%zu)", nmsg);
    if (tile_blocks == 0) return fail(AES_ERR_ARG, "tile size is zero");
    for (size_t i = 0; i < nctx; ++i)
        if (!ctxs[i] || ctxs[i]->magic != kCtxMagic) return fail(AES_ERR_ARG, "ctxs[%zu] is not a valid aes_ctx", i);
    std::vector<uint32_t> order[kGroups];
    for (size_t i = 0; i < nmsg; ++i) {
        const aes_msg_desc& m = d[i];
        if (m.key_index >= nctx) return fail(AES_ERR_ARG, "message %zu: key_index %u >= %zu", i, m.key_index, nctx);
        if (m.decrypt > 1) return fail(AES_ERR_ARG, "message %zu: decrypt must be 0 or 1", i);
        if ((m.in_off | m.out_off) & 15u) return fail(AES_ERR_ALIGN, "message %zu: offsets must be multiples of 16", i);
        if (m.nblocks > (UINT64_MAX >> 5)) return fail(AES_ERR_ARG, "message %zu: nblocks too large", i);
        const uint64_t bytes = m.nblocks * 16;
        if (m.in_off > UINT64_MAX - bytes || m.out_off > UINT64_MAX - bytes)
            return fail(AES_ERR_ARG, "message %zu: offset + length overflows", i);
        if (m.nblocks == 0) continue;
        P->in_extent = std::max<uint64_t>(P->in_extent, m.in_off + bytes);
        P->out_extent = std::max<uint64_t>(P->out_extent, m.out_off + bytes);
        order[group_of(ctxs[m.key_index]->nr, (int)m.decrypt)].push_back((uint32_t)i);
    }
    P->tile_blocks = tile_blocks;
    uint64_t tiles = 0;
    for (int g = 0; g < kGroups; ++g) {
        GroupDev& G = P->groups[g];
        G.nr = g % 3 == 0 ? 10 : g % 3 == 1 ? 12 : 14;
        G.dir = g / 3;
        G.msg_start = (uint32_t)P->msgs.size();
        uint64_t blk = 0;
        for (uint32_t i : order[g]) {
            const aes_msg_desc& m = d[i];
            MsgDev md;
            md.blk_start = blk;
            md.in_blk = m.in_off >> 4;
            md.out_blk = m.out_off >> 4;
            md.key_slot = 2u * m.key_index + m.decrypt;
            md.src = i;
            P->msgs.push_back(md);
            blk += m.nblocks;
        }
        G.msg_end = (uint32_t)P->msgs.size();
        G.blocks = blk;
        const uint64_t gt = (blk + tile_blocks - 1) / tile_blocks;
        // headroom: warps read the counter past the last tile, offset by the fixed first tiles
        if (tiles + gt > 0xFFFF0000u) return fail(AES_ERR_ARG, "batch needs too many tiles");
        G.tile_start = (uint32_t)tiles;
        G.tile_end = (uint32_t)(tiles + gt);
        // first message of each tile: walk the group's messages once
        uint32_t m = G.msg_start;
        for (uint64_t lt = 0; lt < gt; ++lt) {
            const uint64_t first = lt * tile_blocks;
            while (m + 1 < G.msg_end && P->msgs[m + 1].blk_start <= first) ++m;
            P->tile_msg.push_back(m);
        }
        tiles += gt;
        P->total_blocks += blk;
    }
    P->ntiles = (uint32_t)tiles;
    if (with_keys) {
        P->keys.assign(2 * nctx * kSlotWords, 0u);
        for (size_t i = 0; i < nctx; ++i) {
            const int words = 4 * (ctxs[i]->nr + 1);
            memcpy(&P->keys[(2 * i) * kSlotWords], ctxs[i]->enc_rk, 4 * words);
            memcpy(&P->keys[(2 * i + 1) * kSlotWords], ctxs[i]->dec_rk, 4 * words);
        }
    }
    return AES_OK;
}

}  // namespace gbaes

using namespace gbaes;

struct aes_batch_plan {
    uint32_t magic;
    int device;
    int threads, bpt;
    HostPlan host;
    uint8_t* dev_buf;
    size_t dev_bytes;
    BatchArgs args;  // device pointers filled in; in/out set per launch
    cudaGraphExec_t graph_exec;
    cudaGraph_t graph;
    cudaGraphNode_t kernel_node;
    cudaStream_t capture_stream;
    std::mutex mu;
};

namespace gbaes {

constexpr uint32_t kPlanMagic = 0x504c414eu;  // "PLAN"

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

using BatchKernel = void (*)(const BatchArgs);

static BatchKernel pick_batch(int bpt) {
    switch (bpt) {
        case 1: return batch_kernel<1>;
        case 2: return batch_kernel<2>;
        case 4: return batch_kernel<4>;
        case 8: return batch_kernel<8>;  // (512 threads at most: 128 registers per thread)
        default: return nullptr;
    }
}


static int check_bases(const HostPlan& H, const void* in_base, size_t in_bytes, const void* out_base,
                       size_t out_bytes) {
    if (in_bytes < H.in_extent || out_bytes < H.out_extent)
        return fail(AES_ERR_ARG, "buffers (%zu in, %zu out bytes) are smaller than the messages need (%llu, %llu)",
                    in_bytes, out_bytes, (unsigned long long)H.in_extent, (unsigned long long)H.out_extent);
    if (H.ntiles) {
        int rc = check_device_range(in_base, H.in_extent, "in_base");
        if (rc) return rc;
        rc = check_device_range(out_base, H.out_extent, "out_base");
        if (rc) return rc;
    }
    return AES_OK;
}

static int plan_launch_args(aes_batch_plan* P, const void* in_base, size_t in_bytes, void* out_base,
                            size_t out_bytes, BatchArgs* a) {
    if (!P || P->magic != kPlanMagic) return fail(AES_ERR_ARG, "invalid aes_batch_plan");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device)
        return fail(AES_ERR_ARG, "plan was built on device %d, current device is %d", P->device, dev);
    int rc = check_bases(P->host, in_base, in_bytes, out_base, out_bytes);
    if (rc) return rc;
    *a = P->args;
    a->in = (const uint4*)in_base;
    a->out = (uint4*)out_base;
    return AES_OK;
}

// The whole opt-in shared memory (the attribute is set once per kernel and context).
static int batch_smem(BatchKernel fn, int* smem) {
    DeviceInfo info;
    int rc = current_device_info(&info);
    if (rc) return rc;
    rc = set_max_dynamic_smem((const void*)fn, info.smem_optin);
    if (rc) return rc;
    *smem = info.smem_optin;
    return AES_OK;
}

static unsigned batch_grid(uint32_t ntiles) {
    DeviceInfo info;
    if (current_device_info(&info)) return 1;
    return (unsigned)std::min<uint64_t>(ntiles, (uint64_t)info.sms);
}

int launch_batch_kernel(const BatchArgs& a, int threads, int bpt, cudaStream_t stream) {
    BatchKernel fn = pick_batch(bpt);
    if (!fn) return fail(AES_ERR_ARG, "blocks_per_thread %d: need 1, 2, 4 or 8", bpt);
    if (bpt == 8 && threads > 512) return fail(AES_ERR_ARG, "8 blocks per thread need threads <= 512");
    int smem = 0;
    int rc = batch_smem(fn, &smem);
    if (rc) return rc;
    fn<<<batch_grid(a.ntiles), threads, smem, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "batch kernel launch: %s", cudaGetErrorString(e));
    return AES_OK;
}

}  // namespace gbaes

extern "C" {

aes_batch_plan* aes_batch_plan_create(const aes_msg_desc* msgs, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx,
                                      int threads, int blocks_per_thread) {
    if (threads == 0) threads = 1024;
    if (blocks_per_thread == 0) blocks_per_thread = 2;
    if (threads < 64 || threads > 1024 || threads % 32) {
        fail(AES_ERR_ARG, "threads %d: need a multiple of 32 in [64, 1024]", threads);
        return nullptr;
    }
    if (!pick_batch(blocks_per_thread)) {
        fail(AES_ERR_ARG, "blocks_per_thread %d: need 1, 2, 4 or 8", blocks_per_thread);
        return nullptr;
    }
    if (blocks_per_thread == 8 && threads > 512) {
        fail(AES_ERR_ARG, "8 blocks per thread need threads <= 512 (128 registers per thread)");
        return nullptr;
    }
    aes_batch_plan* P = new (std::nothrow) aes_batch_plan();
    if (!P) {
        fail(AES_ERR_NOMEM, "out of host memory");
        return nullptr;
    }
    P->threads = threads;
    P->bpt = blocks_per_thread;
    // Tiles of 128*BPT blocks, at most 512.  A batch of 10,000 messages (16 B - 4 MiB, log-uniform) ran at
    // 0.8847 of its lookup roofline with 1,024-block tiles at 8 blocks per thread and at 0.8878 with 512
    // (less work left over in the last wave); at 4 blocks per thread 256-block tiles lost (0.8705 against
    // 0.8745 at 512).
    const uint32_t tile_blocks = std::min(128u * (uint32_t)blocks_per_thread, kPlanTileMax);
    if (build_host_plan(msgs, nmsg, ctxs, nctx, tile_blocks, true, &P->host)) {
        delete P;
        return nullptr;
    }
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        fail(AES_ERR_CUDA, "no CUDA device");
        delete P;
        return nullptr;
    }
    const HostPlan& H = P->host;
    const size_t off_keys = 256;
    const size_t off_msgs = off_keys + align256(H.keys.size() * 4);
    const size_t off_tiles = off_msgs + align256(H.msgs.size() * sizeof(MsgDev));
    P->dev_bytes = off_tiles + align256(H.tile_msg.size() * 4 + 4);
    cudaError_t e = cudaMalloc(&P->dev_buf, P->dev_bytes);
    if (e != cudaSuccess) {
        fail(AES_ERR_NOMEM, "cudaMalloc(%zu): %s", P->dev_bytes, cudaGetErrorString(e));
        delete P;
        return nullptr;
    }
    std::vector<uint8_t> img(P->dev_bytes, 0);
    if (!H.keys.empty()) memcpy(img.data() + off_keys, H.keys.data(), H.keys.size() * 4);
    if (!H.msgs.empty()) memcpy(img.data() + off_msgs, H.msgs.data(), H.msgs.size() * sizeof(MsgDev));
    if (!H.tile_msg.empty()) memcpy(img.data() + off_tiles, H.tile_msg.data(), H.tile_msg.size() * 4);
    e = cudaMemcpy(P->dev_buf, img.data(), P->dev_bytes, cudaMemcpyHostToDevice);
    int* status = nullptr;
    if (e != cudaSuccess || device_status_word(&status)) {
        fail(AES_ERR_CUDA, "uploading the batch plan: %s", cudaGetErrorString(e));
        cudaFree(P->dev_buf);
        delete P;
        return nullptr;
    }
    BatchArgs& a = P->args;
    memset(&a, 0, sizeof a);
    a.msgs = (const MsgDev*)(P->dev_buf + off_msgs);
    a.keys = (const uint4*)(P->dev_buf + off_keys);
    a.tile_msg = (const uint32_t*)(P->dev_buf + off_tiles);
    a.counter = (unsigned*)P->dev_buf;
    a.status = status;
    a.ntiles = H.ntiles;
    a.tile_blocks = H.tile_blocks;
    memcpy(a.groups, H.groups, sizeof a.groups);
    P->magic = kPlanMagic;
    return P;
}

int aes_batch_plan_launch(aes_batch_plan* P, const void* in_base, size_t in_bytes, void* out_base, size_t out_bytes,
                          void* stream) {
    BatchArgs a;
    int rc = plan_launch_args(P, in_base, in_bytes, out_base, out_bytes, &a);
    if (rc) return rc;
    if (P->host.ntiles == 0) return AES_OK;
    BatchKernel fn = pick_batch(P->bpt);
    int smem = 0;
    rc = batch_smem(fn, &smem);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "resetting the tile counter: %s", cudaGetErrorString(e));
    fn<<<batch_grid(P->host.ntiles), P->threads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "batch kernel launch: %s", cudaGetErrorString(e));
    return AES_OK;
}

int aes_batch_plan_launch_graph(aes_batch_plan* P, const void* in_base, size_t in_bytes, void* out_base,
                                size_t out_bytes, void* stream) {
    BatchArgs a;
    int rc = plan_launch_args(P, in_base, in_bytes, out_base, out_bytes, &a);
    if (rc) return rc;
    if (P->host.ntiles == 0) return AES_OK;
    std::lock_guard<std::mutex> lk(P->mu);
    BatchKernel fn = pick_batch(P->bpt);
    int smem = 0;
    rc = batch_smem(fn, &smem);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (!P->graph_exec) {
        if (!P->capture_stream) {
            e = cudaStreamCreateWithFlags(&P->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return fail(AES_ERR_CUDA, "capture stream: %s", cudaGetErrorString(e));
        }
        e = cudaStreamBeginCapture(P->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(a.counter, 0, 2 * sizeof(unsigned), P->capture_stream);
            fn<<<batch_grid(P->host.ntiles), P->threads, smem, P->capture_stream>>>(a);
            e = cudaStreamEndCapture(P->capture_stream, &P->graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->graph_exec, P->graph, 0);
        if (e == cudaSuccess) {
            size_t n = 0;
            cudaGraphGetNodes(P->graph, nullptr, &n);
            std::vector<cudaGraphNode_t> nodes(n);
            cudaGraphGetNodes(P->graph, nodes.data(), &n);
            for (auto node : nodes) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(node, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                    P->kernel_node = node;
            }
        }
        if (e != cudaSuccess || !P->kernel_node) {
            cudaGetLastError();
            return fail(AES_ERR_CUDA, "capturing the batch graph: %s", cudaGetErrorString(e));
        }
    } else {
        void* params[1] = {&a};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = (void*)fn;
        kp.gridDim = dim3(batch_grid(P->host.ntiles));
        kp.blockDim = dim3(P->threads);
        kp.sharedMemBytes = smem;
        kp.kernelParams = params;
        e = cudaGraphExecKernelNodeSetParams(P->graph_exec, P->kernel_node, &kp);
        if (e != cudaSuccess) return fail(AES_ERR_CUDA, "updating the batch graph: %s", cudaGetErrorString(e));
    }
    e = cudaGraphLaunch(P->graph_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return AES_OK;
}

int aes_batch_plan_info(const aes_batch_plan* P, uint64_t* total_blocks, uint32_t* ntiles, uint32_t* tile_blocks) {
    if (!P || P->magic != kPlanMagic) return fail(AES_ERR_ARG, "invalid aes_batch_plan");
    if (total_blocks) *total_blocks = P->host.total_blocks;
    if (ntiles) *ntiles = P->host.ntiles;
    if (tile_blocks) *tile_blocks = P->host.tile_blocks;
    return AES_OK;
}

void aes_batch_plan_free(aes_batch_plan* P) {
    if (!P || P->magic != kPlanMagic) return;
    P->magic = 0;
    if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->capture_stream) cudaStreamDestroy(P->capture_stream);
    cudaFree(P->dev_buf);
    delete P;
}

int aes_ecb_batch(const aes_msg_desc* msgs, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx, const void* in_base,
                  size_t in_bytes, void* out_base, size_t out_bytes, void* stream) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(AES_ERR_STATE,
                    "aes_ecb_batch uploads from host memory freed on return and cannot be captured; "
                    "use aes_batch_plan_launch_graph");
    HostPlan H;
    int rc = build_host_plan(msgs, nmsg, ctxs, nctx, 2048, true, &H);
    if (rc) return rc;
    if (H.ntiles == 0) return AES_OK;
    rc = check_bases(H, in_base, in_bytes, out_base, out_bytes);
    if (rc) return rc;
    // Stream-ordered scratch: plan tables live only as long as the launch.
    cudaStream_t s = (cudaStream_t)stream;
    const size_t off_keys = 256;
    const size_t off_msgs = off_keys + align256(H.keys.size() * 4);
    const size_t off_tiles = off_msgs + align256(H.msgs.size() * sizeof(MsgDev));
    const size_t bytes = off_tiles + align256(H.tile_msg.size() * 4 + 4);
    std::vector<uint8_t> img(bytes, 0);
    memcpy(img.data() + off_keys, H.keys.data(), H.keys.size() * 4);
    memcpy(img.data() + off_msgs, H.msgs.data(), H.msgs.size() * sizeof(MsgDev));
    memcpy(img.data() + off_tiles, H.tile_msg.data(), H.tile_msg.size() * 4);
    uint8_t* buf = nullptr;
    e = cudaMallocAsync((void**)&buf, bytes, s);
    if (e != cudaSuccess) return fail(AES_ERR_NOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    e = cudaMemcpyAsync(buf, img.data(), bytes, cudaMemcpyHostToDevice, s);  // pageable: staged before return
    int* status = nullptr;
    if (e != cudaSuccess || device_status_word(&status)) {
        cudaFreeAsync(buf, s);
        return fail(AES_ERR_CUDA, "uploading the batch tables: %s", cudaGetErrorString(e));
    }
    BatchArgs a;
    memset(&a, 0, sizeof a);
    a.in = (const uint4*)in_base;
    a.out = (uint4*)out_base;
    a.msgs = (const MsgDev*)(buf + off_msgs);
    a.keys = (const uint4*)(buf + off_keys);
    a.tile_msg = (const uint32_t*)(buf + off_tiles);
    a.counter = (unsigned*)buf;
    a.status = status;
    a.ntiles = H.ntiles;
    a.tile_blocks = H.tile_blocks;
    memcpy(a.groups, H.groups, sizeof a.groups);
    BatchKernel fn = pick_batch(2);
    int smem = 0;
    rc = batch_smem(fn, &smem);
    if (rc) {
        cudaFreeAsync(buf, s);
        return rc;
    }
    fn<<<batch_grid(H.ntiles), 1024, smem, s>>>(a);
    e = cudaGetLastError();
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "batch kernel launch: %s", cudaGetErrorString(e));
    return AES_OK;
}

int aes_batch_tiles(const aes_msg_desc* msgs, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx, int tile_blocks,
                    uint32_t* first_msg, size_t cap) {
    if (tile_blocks <= 0) return fail(AES_ERR_ARG, "tile_blocks must be positive");
    HostPlan H;
    int rc = build_host_plan(msgs, nmsg, ctxs, nctx, (uint32_t)tile_blocks, false, &H);
    if (rc) return rc;
    if (first_msg) {
        if (cap < H.ntiles) return fail(AES_ERR_ARG, "first_msg holds %zu entries, the batch has %u tiles", cap, H.ntiles);
        for (uint32_t t = 0; t < H.ntiles; ++t) first_msg[t] = H.msgs[H.tile_msg[t]].src;
    }
    return (int)std::min<uint32_t>(H.ntiles, 0x7FFFFFFF);
}

}  // extern "C"

// ------------------------------------------------ batch without allocation
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another runtime or allocator (a cudaMalloc behind its back breaks its
// accounting, or fails once it has reserved the device), and latency-critical
// paths that must not pay an allocation's synchronisation or unbounded cost.
// aes_ecb_batch_noalloc serves them: it runs the same batched kernel as
// aes_ecb_batch, but its plan tables and tile counter live in the fixed array
// below, which every GPU that loads this library holds until the process exits.

namespace gbaes {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // 8 MiB

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static std::vector<std::pair<unsigned long long, uint8_t*>> g_noalloc_addr;  // (context id, device address)

// Device address of g_noalloc_scratch in the current context.  Host code must
// not pass the array's own name to a kernel: on the host that name denotes a
// host-side stand-in, not device memory.  The address belongs to the module
// loaded in one CUDA context, so it is looked up (cudaGetSymbolAddress, with
// that context current) on the first call in each context -- normally once per
// device, in its primary context -- and cached under the context's id.
static int noalloc_scratch(uint8_t** out) {
    unsigned long long ctx = 0;
    int rc = current_context_id(&ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (const auto& e : g_noalloc_addr)
        if (e.first == ctx) {
            *out = e.second;
            return AES_OK;
        }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(AES_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_addr.emplace_back(ctx, (uint8_t*)p);
    *out = (uint8_t*)p;
    return AES_OK;
}

}  // namespace gbaes

extern "C" {

int aes_ecb_batch_noalloc(const aes_msg_desc* msgs, size_t nmsg, const aes_ctx* const* ctxs, size_t nctx,
                          const void* in_base, size_t in_bytes, void* out_base, size_t out_bytes, void* stream) {
    HostPlan H;
    int rc = build_host_plan(msgs, nmsg, ctxs, nctx, 2048, true, &H);
    if (rc) return rc;
    if (H.ntiles == 0) return AES_OK;
    rc = check_bases(H, in_base, in_bytes, out_base, out_bytes);
    if (rc) return rc;
    const size_t off_keys = 256;  // [0, 256): tile counter, uploaded as zero
    const size_t off_msgs = off_keys + align256(H.keys.size() * 4);
    const size_t off_tiles = off_msgs + align256(H.msgs.size() * sizeof(MsgDev));
    const size_t bytes = off_tiles + align256(H.tile_msg.size() * 4 + 4);
    if (bytes > kNoAllocScratchBytes)
        return fail(AES_ERR_ARG,
                    "batch needs %zu bytes of tables (keys: 512 B per context; 32 B per message; 4 B per tile), "
                    "the allocation-free entry point holds at most %zu",
                    bytes, kNoAllocScratchBytes);
    uint8_t* buf = nullptr;
    rc = noalloc_scratch(&buf);
    if (rc) return rc;
    int* status = nullptr;
    rc = device_status_word(&status);
    if (rc) return rc;
    BatchKernel fn = pick_batch(2);
    int smem = 0;
    rc = batch_smem(fn, &smem);
    if (rc) return rc;
    std::vector<uint8_t> img(bytes, 0);  // host staging only; the counter word stays zero
    memcpy(img.data() + off_keys, H.keys.data(), H.keys.size() * 4);
    memcpy(img.data() + off_msgs, H.msgs.data(), H.msgs.size() * sizeof(MsgDev));
    memcpy(img.data() + off_tiles, H.tile_msg.data(), H.tile_msg.size() * 4);
    cudaStream_t s = (cudaStream_t)stream;
    // Stream-ordered after earlier work on `stream`; from pageable memory the
    // call returns once the image is staged, so img may be released after it.
    cudaError_t e = cudaMemcpyAsync(buf, img.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "uploading the batch tables: %s", cudaGetErrorString(e));
    BatchArgs a;
    memset(&a, 0, sizeof a);
    a.in = (const uint4*)in_base;
    a.out = (uint4*)out_base;
    a.msgs = (const MsgDev*)(buf + off_msgs);
    a.keys = (const uint4*)(buf + off_keys);
    a.tile_msg = (const uint32_t*)(buf + off_tiles);
    a.counter = (unsigned*)buf;
    a.status = status;
    a.ntiles = H.ntiles;
    a.tile_blocks = H.tile_blocks;
    memcpy(a.groups, H.groups, sizeof a.groups);
    fn<<<batch_grid(H.ntiles), 1024, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "batch kernel launch: %s", cudaGetErrorString(e));
    return AES_OK;
}

}  // extern "C"
