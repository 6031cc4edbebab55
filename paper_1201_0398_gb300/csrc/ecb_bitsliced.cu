// Bitsliced AES-ECB kernel (the Boolean-circuit alternative to Eq. 1's tables).
//
// A pair of lanes holds 32 blocks as 128 bit planes (bitsliced.h), split by
// state columns: lane 2g+h holds the 64 planes of columns 2h and 2h+1 of the 32
// blocks of its pair g.  A warp takes 512 consecutive blocks: pair g owns
// blocks base + 16k + g (k = 0..31) and lane h loads bytes 8h..8h+15 of each
// with a coalesced 8-byte load (the warp reads 256 contiguous bytes per load),
// transposes its two 32x32 bit matrices in registers, runs the rounds as
// bitwise logic with no memory lookups (ShiftRows trades four bytes' planes
// with the other lane of the pair by shuffle; the S-box and the column maps as
// generated LOP3 programs), transposes back and stores.
// Splitting the state halves the registers a lane needs (four CTAs of 128
// threads per SM instead of two; five for encryption, whose column map is
// smaller and fits 96 registers) and the unrolled round body each lane runs.
// Round-key planes (0 or all ones, the S-box's affine constant folded in) are
// staged once per CTA in shared memory, each half's row in its own banks.  The
// kernel is bound by the integer pipe, not by shared memory: it is the measured
// counterpart to the T-table kernel.
#include <mutex>

#include "bitsliced.h"
#include "gbaes_internal.h"

namespace gbaes {

constexpr int kBsThreads = 128;
constexpr int kBsCtasPerSmEnc = 5;  // 96 registers per thread (20 warps per SM)
constexpr int kBsCtasPerSmDec = 4;  // 128 registers per thread
constexpr int kBsWarpBlocks = 512;  // 16 lane pairs x 32 blocks

struct BsArgs {
    const uint4* in;
    uint4* out;
    uint64_t nblocks;
    uint32_t planes[15 * bs::kKeyStepWords];  // split_key_planes layout (8,160 bytes)
};

// The other lane of the pair (lane ^ 1) hands over its copy of the plane.
struct PairShuffle {
    __device__ uint32_t operator()(uint32_t v, int) const { return __shfl_xor_sync(0xffffffffu, v, 1); }
};

template <int NR, bool DEC>
__global__ void __launch_bounds__(kBsThreads, DEC ? kBsCtasPerSmDec : kBsCtasPerSmEnc)
    bitsliced_kernel(const __grid_constant__ BsArgs a) {
    __shared__ __align__(16) uint32_t keys_s[(NR + 1) * bs::kKeyStepWords];
    for (int i = threadIdx.x; i < (NR + 1) * bs::kKeyStepWords; i += blockDim.x) keys_s[i] = a.planes[i];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t h = lane & 1u, g = lane >> 1;
    const bs::HalfKeys keys{keys_s + bs::kKeyHalfWords * h};
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = warp * kBsWarpBlocks; base < a.nblocks; base += nwarps * kBsWarpBlocks) {
        uint32_t s[64];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint64_t idx = base + 16u * k + g;
            uint2 v = make_uint2(0, 0);
            if (idx < a.nblocks) v = __ldcs(reinterpret_cast<const uint2*>(a.in + idx) + h);
            s[k] = v.x;
            s[32 + k] = v.y;
        }
        bs::transpose32(&s[0]);  // s[32i + j] = bit j of word 2h + i: local plane 32i + j
        bs::transpose32(&s[32]);
        if (DEC)
            bs::decrypt_half<NR>(s, keys, PairShuffle{});
        else
            bs::encrypt_half<NR>(s, keys, PairShuffle{});
        bs::transpose32(&s[0]);
        bs::transpose32(&s[32]);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint64_t idx = base + 16u * k + g;
            if (idx < a.nblocks) __stcs(reinterpret_cast<uint2*>(a.out + idx) + h, make_uint2(s[k], s[32 + k]));
        }
    }
}

namespace {

using BsKernel = void (*)(const BsArgs);

BsKernel pick_bs(int nr, bool dec) {
    switch (nr * 2 + (dec ? 1 : 0)) {
        case 20: return bitsliced_kernel<10, false>;
        case 21: return bitsliced_kernel<10, true>;
        case 24: return bitsliced_kernel<12, false>;
        case 25: return bitsliced_kernel<12, true>;
        case 28: return bitsliced_kernel<14, false>;
        case 29: return bitsliced_kernel<14, true>;
        default: return nullptr;
    }
}

}  // namespace

int launch_bitsliced(const EcbArgs& e, const uint32_t* enc_rk, int nr, Mode mode, int threads, cudaStream_t stream) {
    if (mode != kEnc && mode != kDec) return fail(AES_ERR_ARG, "the bitsliced kernel implements ECB only");
    const bool dec = mode == kDec;
    BsKernel fn = pick_bs(nr, dec);
    if (!fn) return fail(AES_ERR_ARG, "no bitsliced kernel for nr=%d", nr);
    (void)threads;  // the kernel's shape is fixed by its register budget: 128 threads, 4-5 CTAs per SM
    static BsArgs a;  // 8.2 KB: built here, copied into the launch by value
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    a.in = e.in;
    a.out = e.out;
    a.nblocks = e.nblocks;
    uint32_t planes[15][128];
    bs::make_key_planes(enc_rk, nr, dec, planes);
    bs::split_key_planes(planes, nr, a.planes);
    DeviceInfo info;
    int rc = current_device_info(&info);
    if (rc) return rc;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBsThreads, 0);
    if (err != cudaSuccess || per_sm < 1) per_sm = 1;
    const uint64_t tiles = (e.nblocks + kBsWarpBlocks - 1) / kBsWarpBlocks;
    const uint64_t warps_per_cta = kBsThreads / 32;
    uint64_t grid = (uint64_t)info.sms * per_sm;
    const uint64_t need = (tiles + warps_per_cta - 1) / warps_per_cta;
    if (need < grid) grid = need;
    fn<<<(unsigned)grid, kBsThreads, 0, stream>>>(a);
    err = cudaGetLastError();
    if (err != cudaSuccess) return fail(AES_ERR_CUDA, "bitsliced kernel launch: %s", cudaGetErrorString(err));
    return AES_OK;
}

}  // namespace gbaes
