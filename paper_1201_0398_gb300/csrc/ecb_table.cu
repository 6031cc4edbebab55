// T-table AES kernels for sm_103a: ECB encryption/decryption, CTR, CBC decryption.
//
// Each round is Eq. 1 of the paper: four output words, each the XOR of four
// 32-bit table lookups and a round-key word,
//     O_j = T0[I_{j,0}] ^ T1[I_{j+1,1}] ^ T2[I_{j+2,2}] ^ T3[I_{j+3,3}] ^ K_j
// (indices of I mod 4), and for the inverse cipher the same with Td tables and
// I_{j-k,k}.  The paper keeps the tables in a texture (Section 3); here they sit
// in shared memory in the conflict-free, one-PRMT-per-address layout described
// in aes_rounds.cuh, 128 KiB (encryption) or 160 KiB (decryption) per CTA.
//
// One CTA per SM (the tables fill most of the SM's shared memory), persistent
// over the input in tiles of threads*BPT blocks; each block is a coalesced
// 16-byte load and store, and round keys come from the kernel parameters.
#include "aes_rounds.cuh"

namespace gbaes {

__device__ int g_status;  // nonzero: a kernel found that its shared-memory layout did not fit

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123u); }

// Counter block for counter index i (128-bit base + i, modulo 2^128).
__device__ __forceinline__ void counter_words(const EcbArgs& a, uint64_t i, uint32_t (&w)[4]) {
    uint64_t lo = a.ctr_lo + i;
    uint64_t hi = a.ctr_hi + (lo < a.ctr_lo ? 1u : 0u);
    if (a.ctr_be) {
        w[0] = bswap32((uint32_t)(hi >> 32));
        w[1] = bswap32((uint32_t)hi);
        w[2] = bswap32((uint32_t)(lo >> 32));
        w[3] = bswap32((uint32_t)lo);
    } else {
        w[0] = (uint32_t)lo;
        w[1] = (uint32_t)(lo >> 32);
        w[2] = (uint32_t)hi;
        w[3] = (uint32_t)(hi >> 32);
    }
}

template <int NR, int MODE, int BPT>
__global__ void __launch_bounds__(1024, 1) table_kernel(const EcbArgs a) {
    constexpr bool DECRYPT = (MODE == kDec || MODE == kCbcDec);
    constexpr uint32_t kNeed = DECRYPT ? kDecBytes : kEncBytes;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t base = smem_base(smem_raw);
    const uint32_t A = table_base(base);
    if (A + kNeed > base + dynamic_smem_bytes()) {  // same outcome in every thread of every CTA
        if (threadIdx.x == 0) atomicOr(&g_status, 1);
        return;
    }
    fill_tables(A, DECRYPT);
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t L0 = A | (lane << 2);
    const uint32_t L1 = L0 | 128u;
    const uint64_t n = a.nblocks;
    const uint64_t tile = (uint64_t)blockDim.x * BPT;
    const uint64_t stride = (uint64_t)gridDim.x * tile;

    for (uint64_t t0b = (uint64_t)blockIdx.x * tile; t0b < n; t0b += stride) {
        if (t0b + threadIdx.x >= n) break;  // no block left for this thread (only the last tile is partial)
        uint32_t s[BPT][4];
        uint4 aux[BPT];  // CTR: data; CBC: previous ciphertext block
        uint64_t idx[BPT];
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            idx[b] = t0b + threadIdx.x + (uint64_t)b * blockDim.x;
            const bool ok = idx[b] < n;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (MODE == kCtr) {
                counter_words(a, a.first + idx[b], s[b]);
                if (ok) v = ld_stream(a.in + idx[b]);
                aux[b] = v;
            } else {
                if (ok) v = ld_stream(a.in + idx[b]);
                s[b][0] = v.x;
                s[b][1] = v.y;
                s[b][2] = v.z;
                s[b][3] = v.w;
                if (MODE == kCbcDec) {
                    uint4 p = make_uint4(a.iv[0], a.iv[1], a.iv[2], a.iv[3]);
                    if (ok && idx[b] > 0) p = __ldg(a.in + idx[b] - 1);
                    aux[b] = p;
                }
            }
        }
        cipher<NR, DECRYPT, BPT>(s, ParamKeys{a.rk}, L0, L1);
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            if (idx[b] < n) {
                uint4 o = make_uint4(s[b][0], s[b][1], s[b][2], s[b][3]);
                if (MODE == kCtr || MODE == kCbcDec) {
                    o.x ^= aux[b].x;
                    o.y ^= aux[b].y;
                    o.z ^= aux[b].z;
                    o.w ^= aux[b].w;
                }
                __stcs(a.out + idx[b], o);
            }
        }
    }
}

// ------------------------------------------------------------------ launcher

}  // namespace gbaes

namespace gbaes {

namespace {

using KernelFn = void (*)(const EcbArgs);

template <int NR, int MODE>
KernelFn pick_bpt(int bpt) {
    switch (bpt) {
        case 1: return table_kernel<NR, MODE, 1>;
        case 2: return table_kernel<NR, MODE, 2>;
        case 4: return table_kernel<NR, MODE, 4>;
        default: return nullptr;
    }
}

template <int NR>
KernelFn pick_mode(int mode, int bpt) {
    switch (mode) {
        case kEnc: return pick_bpt<NR, kEnc>(bpt);
        case kDec: return pick_bpt<NR, kDec>(bpt);
        case kCtr: return pick_bpt<NR, kCtr>(bpt);
        case kCbcDec: return pick_bpt<NR, kCbcDec>(bpt);
        default: return nullptr;
    }
}

KernelFn pick(int nr, int mode, int bpt) {
    switch (nr) {
        case 10: return pick_mode<10>(mode, bpt);
        case 12: return pick_mode<12>(mode, bpt);
        case 14: return pick_mode<14>(mode, bpt);
        default: return nullptr;
    }
}

}  // namespace

int launch_table(const EcbArgs& a, int nr, Mode mode, int threads, int bpt, cudaStream_t stream) {
    KernelFn fn = pick(nr, mode, bpt);
    if (!fn) return fail(AES_ERR_ARG, "no table kernel for nr=%d mode=%d blocks_per_thread=%d", nr, (int)mode, bpt);
    DeviceInfo info;
    int rc = current_device_info(&info);
    if (rc) return rc;
    // Dynamic shared memory: the whole opt-in limit, so the 64 KiB-aligned
    // layout fits wherever the dynamic window starts (the kernel re-checks).
    const int smem = info.smem_optin;
    rc = set_max_dynamic_smem((const void*)fn, smem);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    // Small inputs: no more threads than blocks to process (a whole warp at least).
    const uint64_t need_threads = ((a.nblocks + bpt - 1) / bpt + 31) / 32 * 32;
    if (need_threads < (uint64_t)threads) threads = (int)(need_threads < 64 ? 64 : need_threads);
    const uint64_t per_cta = (uint64_t)threads * (uint64_t)bpt;
    const uint64_t want = (a.nblocks + per_cta - 1) / per_cta;
    const unsigned grid = (unsigned)(want < (uint64_t)info.sms ? want : (uint64_t)info.sms);
    fn<<<grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "table kernel launch: %s", cudaGetErrorString(e));
    return AES_OK;
}

int device_status_word(int** p) {
    cudaError_t e = cudaGetSymbolAddress((void**)p, g_status);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "status word address: %s", cudaGetErrorString(e));
    return AES_OK;
}

int read_device_status(int clear) {
    int v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_status, sizeof(int));
    if (e == cudaSuccess && clear) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
    }
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "reading device status: %s", cudaGetErrorString(e));
    return v;
}

}  // namespace gbaes
