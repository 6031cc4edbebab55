// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "gbaes.h"

struct aes_ctx {
    uint32_t magic;
    int bits;
    int nr;
    uint32_t enc_rk[60];  // 4*(Nr+1) words; word j of round r at [4r+j]
    uint32_t dec_rk[60];  // equivalent inverse cipher schedule
};

namespace gbaes {

constexpr uint32_t kCtxMagic = 0x41455343u;  // "AESC"

// Error recording (thread-local message, returned code).
int fail(int code, const char* fmt, ...);
void clear_error();

// Operation performed by the block kernels.
enum Mode : int { kEnc = 0, kDec = 1, kCtr = 2, kCbcDec = 3 };

// Arguments of one block-kernel launch, passed by value (they live in the
// kernel parameter constant bank, so round keys are read as uniform operands).
struct EcbArgs {
    const uint4* in;
    uint4* out;
    uint64_t nblocks;
    uint32_t rk[60];   // encryption schedule (kEnc, kCtr) or decryption schedule (kDec, kCbcDec)
    uint64_t ctr_lo;   // kCtr: 128-bit counter base (low, high halves as integers)
    uint64_t ctr_hi;
    uint64_t first;    // kCtr: counter index of in[0]
    uint32_t iv[4];    // kCbcDec: ciphertext block before in[0]
    int ctr_be;        // kCtr: 1 = big-endian 128-bit counter, 0 = little-endian words
};

struct DeviceInfo {
    int device;
    int sms;
    int smem_optin;           // max dynamic shared memory per block (bytes)
    int pageable_access;      // GPU can read pageable host memory (ATS/HMM)
};

// Cached properties of the current device.  Returns AES_OK or an error code.
int current_device_info(DeviceInfo* info);

// Process-unique id of the CUDA context current on this thread (the device's
// primary context is made current first if none is).
int current_context_id(unsigned long long* id);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) for kernel fn, once per
// (kernel, context).
int set_max_dynamic_smem(const void* fn, int bytes);

// Checks that [p, p+bytes) is 16-byte aligned device-reachable memory.
int check_device_range(const void* p, size_t bytes, const char* what);

// Allocations already found valid during one pass of checks over many ranges
// (which must not free or replace them meanwhile): a range inside one of them
// needs no driver query.
struct RangeCache {
    static constexpr int kSize = 8;
    uintptr_t lo[kSize] = {}, hi[kSize] = {};
    int n = 0;
    unsigned next = 0;
};

// check_device_range through a cache (nullptr: no cache).
int check_device_range_cached(const void* p, size_t bytes, const char* what, RangeCache* cache);

// Largest call (in blocks) that AES_KERNEL_TABLE runs with compact tables.
uint64_t compact_limit_blocks(int sms);

// Launches the T-table kernel (ecb_table.cu).  variant: AES_KERNEL_TABLE (picks
// by size), AES_KERNEL_TABLE_COMPACT or AES_KERNEL_TABLE_REPLICATED; threads
// and bpt shape the replicated kernel only.
int launch_table(const EcbArgs& a, int nr, Mode mode, int threads, int bpt, int variant, cudaStream_t stream);

// Launches the bitsliced kernel (ecb_bitsliced.cu), ECB only.
int launch_bitsliced(const EcbArgs& a, const uint32_t* enc_rk, int nr, Mode mode, int threads, cudaStream_t stream);

// Library status word on the device (set by kernels that detect an error).
int read_device_status(int clear);

}  // namespace gbaes
