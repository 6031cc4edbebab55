// Host <-> device pipeline for data that lives in host memory.
//
// The paper copies each 64 MB texture over PCIe, draws, then maps the result
// back, one step after the other, and finds the copies dominate small inputs
// (Section 3, Fig. 3; Section 3.1).  A pipeline object chooses how host data
// reaches the SMs:
//
//  * staged: it owns `depth` device staging slots, each with its own stream.  A
//    call cuts the host buffer into chunks and deals them round-robin to the
//    slots; on its slot's stream a chunk is copied in by a copy engine,
//    enciphered in place by the table kernel and copied out.  Different slots
//    run concurrently, so the copy-in of one chunk, the kernel of another and
//    the copy-out of a third overlap (the two copy directions use separate copy
//    engines).  A slot is reused only after its stream has finished the
//    previous chunk's copy-out, by stream order.  The caller's stream waits for
//    all slots at the end.
//  * direct: the table kernel loads its input from and stores its output to
//    the page-locked host buffers themselves, over the coherent host link, in
//    one launch on the caller's stream.  No staging memory, no copy engine.  On
//    a Grace-Blackwell node this moves each byte once in each direction, as the
//    copies do, and the SMs keep more requests in flight than the copy engines:
//    it measured 165-170 GB/s where the staged pipeline measured 90-160 GB/s.
//
// Either way the call is asynchronous on the caller's stream like the
// device-memory calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>

#include "gbaes_internal.h"

struct aes_pipeline {
    uint32_t magic;
    int device;
    size_t chunk_bytes;
    int depth;
    int mode;  // AES_PIPE_STAGED or AES_PIPE_DIRECT
    uint8_t* slot_buf[16];
    cudaStream_t slot_stream[16];
    cudaEvent_t slot_done[16];
    cudaEvent_t start;
    std::mutex mu;
};

namespace gbaes {

constexpr uint32_t kPipeMagic = 0x50495045u;  // "PIPE"
constexpr int kMaxDepth = 16;
// Launch shape of the direct mode: 512 threads x 4 blocks per thread keeps 32 KiB
// of loads in flight per SM, enough to cover the host link's latency.
constexpr int kDirectThreads = 512;
constexpr int kDirectBpt = 4;

static void destroy_pipeline(aes_pipeline* P) {
    for (int i = 0; i < kMaxDepth; ++i) {
        if (P->slot_done[i]) cudaEventDestroy(P->slot_done[i]);
        if (P->slot_stream[i]) cudaStreamDestroy(P->slot_stream[i]);
        if (P->slot_buf[i]) cudaFree(P->slot_buf[i]);
    }
    if (P->start) cudaEventDestroy(P->start);
    delete P;
}

int table_default_shape(int bits, int decrypt, int* threads, int* bpt);  // api.cu

}  // namespace gbaes

using namespace gbaes;

extern "C" {

aes_pipeline* aes_pipeline_create_ex(size_t chunk_bytes, int depth, int mode) {
    if (mode != AES_PIPE_STAGED && mode != AES_PIPE_DIRECT) {
        fail(AES_ERR_ARG, "mode %d: need AES_PIPE_STAGED or AES_PIPE_DIRECT", mode);
        return nullptr;
    }
    if (chunk_bytes == 0) chunk_bytes = (size_t)64 << 20;
    if (depth == 0) depth = 4;
    if (chunk_bytes % 16 || chunk_bytes > ((size_t)1 << 40)) {
        fail(AES_ERR_ARG, "chunk_bytes %zu: need a positive multiple of 16", chunk_bytes);
        return nullptr;
    }
    if (depth < 1 || depth > kMaxDepth) {
        fail(AES_ERR_ARG, "depth %d: need 1..%d", depth, kMaxDepth);
        return nullptr;
    }
    aes_pipeline* P = new (std::nothrow) aes_pipeline();
    if (!P) {
        fail(AES_ERR_NOMEM, "out of host memory");
        return nullptr;
    }
    P->chunk_bytes = chunk_bytes;
    P->depth = mode == AES_PIPE_DIRECT ? 0 : depth;
    P->mode = mode;
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess && mode == AES_PIPE_STAGED) e = cudaEventCreateWithFlags(&P->start, cudaEventDisableTiming);
    for (int i = 0; i < P->depth && e == cudaSuccess; ++i) {
        e = cudaMalloc(&P->slot_buf[i], chunk_bytes);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->slot_stream[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->slot_done[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        fail(e == cudaErrorMemoryAllocation ? AES_ERR_NOMEM : AES_ERR_CUDA, "pipeline setup: %s",
             cudaGetErrorString(e));
        cudaGetLastError();
        destroy_pipeline(P);
        return nullptr;
    }
    P->magic = kPipeMagic;
    return P;
}

aes_pipeline* aes_pipeline_create(size_t chunk_bytes, int depth) {
    return aes_pipeline_create_ex(chunk_bytes, depth, AES_PIPE_STAGED);
}

int aes_pipeline_ecb(aes_pipeline* P, const aes_ctx* ctx, int decrypt, const void* host_in, void* host_out,
                     size_t nblocks, void* stream) {
    if (!P || P->magic != kPipeMagic) return fail(AES_ERR_ARG, "invalid aes_pipeline");
    if (!ctx || ctx->magic != kCtxMagic) return fail(AES_ERR_ARG, "invalid or freed aes_ctx");
    if (decrypt != 0 && decrypt != 1) return fail(AES_ERR_ARG, "decrypt must be 0 or 1");
    if (nblocks == 0) return AES_OK;
    if (nblocks > (SIZE_MAX >> 4)) return fail(AES_ERR_ARG, "nblocks %zu overflows the byte count", nblocks);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device)
        return fail(AES_ERR_ARG, "pipeline was built on device %d, current device is %d", P->device, dev);
    const size_t bytes = nblocks * 16;
    int rc = check_device_range(host_in, bytes, "host_in");
    if (rc) return rc;
    rc = check_device_range(host_out, bytes, "host_out");
    if (rc) return rc;
    const uintptr_t i0 = (uintptr_t)host_in, o0 = (uintptr_t)host_out;
    if (i0 != o0 && i0 < o0 + bytes && o0 < i0 + bytes) return fail(AES_ERR_ARG, "host_in and host_out overlap partially");
    EcbArgs a;
    memset(&a, 0, sizeof a);
    memcpy(a.rk, decrypt ? ctx->dec_rk : ctx->enc_rk, sizeof(uint32_t) * 4 * (ctx->nr + 1));
    const Mode mode = decrypt ? kDec : kEnc;
    cudaStream_t user = (cudaStream_t)stream;
    if (P->mode == AES_PIPE_DIRECT) {
        a.in = (const uint4*)host_in;
        a.out = (uint4*)host_out;
        a.nblocks = nblocks;
        return launch_table(a, ctx->nr, mode, kDirectThreads, kDirectBpt, AES_KERNEL_TABLE, user);
    }
    int threads = 1024, bpt = 2;
    table_default_shape(ctx->bits, decrypt, &threads, &bpt);
    std::lock_guard<std::mutex> lk(P->mu);
    cudaError_t e = cudaEventRecord(P->start, user);
    const size_t nchunks = (bytes + P->chunk_bytes - 1) / P->chunk_bytes;
    const int used = (int)std::min<size_t>(nchunks, (size_t)P->depth);
    for (int s = 0; s < used && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(P->slot_stream[s], P->start, 0);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "pipeline start: %s", cudaGetErrorString(e));
    for (size_t c = 0; c < nchunks; ++c) {
        const int s = (int)(c % (size_t)P->depth);
        const size_t off = c * P->chunk_bytes;
        const size_t n = std::min(P->chunk_bytes, bytes - off);
        cudaStream_t st = P->slot_stream[s];
        e = cudaMemcpyAsync(P->slot_buf[s], (const uint8_t*)host_in + off, n, cudaMemcpyDefault, st);
        if (e != cudaSuccess) return fail(AES_ERR_CUDA, "copy in: %s", cudaGetErrorString(e));
        a.in = (const uint4*)P->slot_buf[s];
        a.out = (uint4*)P->slot_buf[s];
        a.nblocks = n / 16;
        rc = launch_table(a, ctx->nr, mode, threads, bpt, AES_KERNEL_TABLE, st);
        if (rc) return rc;
        e = cudaMemcpyAsync((uint8_t*)host_out + off, P->slot_buf[s], n, cudaMemcpyDefault, st);
        if (e != cudaSuccess) return fail(AES_ERR_CUDA, "copy out: %s", cudaGetErrorString(e));
    }
    for (int s = 0; s < used && e == cudaSuccess; ++s) {
        e = cudaEventRecord(P->slot_done[s], P->slot_stream[s]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(user, P->slot_done[s], 0);
    }
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "pipeline join: %s", cudaGetErrorString(e));
    return AES_OK;
}

void aes_pipeline_free(aes_pipeline* P) {
    if (!P || P->magic != kPipeMagic) return;
    P->magic = 0;
    for (int s = 0; s < P->depth; ++s)
        if (P->slot_stream[s]) cudaStreamSynchronize(P->slot_stream[s]);
    destroy_pipeline(P);
}

}  // extern "C"
