// Bitsliced AES-ECB kernel (the Boolean-circuit alternative to Eq. 1's tables).
//
// Each thread holds 32 blocks as 128 bit planes (bitsliced.h): a warp loads
// 1,024 consecutive blocks with coalesced 16-byte loads (lane l takes blocks
// base + 32k + l, k = 0..31), each thread transposes its four 32x32 bit
// matrices in registers, runs the rounds as bitwise logic with no memory
// lookups at all, transposes back and stores.  Round-key planes (0 or all
// ones, the S-box's affine constant folded in) travel in the kernel's large
// parameter block.  The kernel is bound by the integer pipe, not by shared
// memory: it is the measured counterpart to the T-table kernel.
#include <mutex>

#include "bitsliced.h"
#include "gbaes_internal.h"

namespace gbaes {

struct BsArgs {
    const uint4* in;
    uint4* out;
    uint64_t nblocks;
    uint32_t planes[15][128];  // key planes per step (7,680 bytes)
};

template <int NR, bool DEC>
__global__ void __launch_bounds__(128) bitsliced_kernel(const __grid_constant__ BsArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const bs::PlaneKeys keys{a.planes};
    for (uint64_t base = warp * 1024; base < a.nblocks; base += nwarps * 1024) {
        uint32_t s[128];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint64_t idx = base + 32u * k + lane;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (idx < a.nblocks) v = __ldcs(a.in + idx);
            s[k] = v.x;
            s[32 + k] = v.y;
            s[64 + k] = v.z;
            s[96 + k] = v.w;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) bs::transpose32(&s[32 * i]);  // s[32i + j] = plane 32i + j
        if (DEC)
            bs::decrypt_planes<NR>(s, keys);
        else
            bs::encrypt_planes<NR>(s, keys);
#pragma unroll
        for (int i = 0; i < 4; ++i) bs::transpose32(&s[32 * i]);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint64_t idx = base + 32u * k + lane;
            if (idx < a.nblocks) __stcs(a.out + idx, make_uint4(s[k], s[32 + k], s[64 + k], s[96 + k]));
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
    if (threads % 32 || threads < 32 || threads > 128) threads = 128;
    static BsArgs a;  // 7.7 KB: built here, copied into the launch by value
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    a.in = e.in;
    a.out = e.out;
    a.nblocks = e.nblocks;
    bs::make_key_planes(enc_rk, nr, dec, a.planes);
    DeviceInfo info;
    int rc = current_device_info(&info);
    if (rc) return rc;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    if (err != cudaSuccess || per_sm < 1) per_sm = 1;
    const uint64_t tiles = (e.nblocks + 1023) / 1024;  // one warp tile = 1,024 blocks
    const uint64_t warps_per_cta = (uint64_t)threads / 32;
    uint64_t grid = (uint64_t)info.sms * per_sm;
    const uint64_t need = (tiles + warps_per_cta - 1) / warps_per_cta;
    if (need < grid) grid = need;
    fn<<<(unsigned)grid, threads, 0, stream>>>(a);
    err = cudaGetLastError();
    if (err != cudaSuccess) return fail(AES_ERR_CUDA, "bitsliced kernel launch: %s", cudaGetErrorString(err));
    return AES_OK;
}

}  // namespace gbaes
