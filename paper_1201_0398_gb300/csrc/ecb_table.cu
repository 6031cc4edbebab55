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

// Loads block idx of the input (ok: idx < n) into the cipher state s, and what
// the mode combines with the cipher output into aux: CTR encrypts the counter
// block and keeps the data, CBC decryption keeps the previous ciphertext block
// (the IV for block 0).  Lanes past the end compute on zeros.
template <int MODE>
__device__ __forceinline__ void load_block(const EcbArgs& a, uint64_t idx, bool ok, uint32_t (&s)[4], uint4& aux) {
    uint4 v = make_uint4(0, 0, 0, 0);
    if (MODE == kCtr) {
        counter_words(a, a.first + idx, s);
        if (ok) v = ld_stream(a.in + idx);
        aux = v;
    } else {
        if (ok) v = ld_stream(a.in + idx);
        s[0] = v.x;
        s[1] = v.y;
        s[2] = v.z;
        s[3] = v.w;
        if (MODE == kCbcDec) {
            uint4 p = make_uint4(a.iv[0], a.iv[1], a.iv[2], a.iv[3]);
            if (ok && idx > 0) p = __ldg(a.in + idx - 1);
            aux = p;
        }
    }
}

template <int MODE>
__device__ __forceinline__ void store_block(const EcbArgs& a, uint64_t idx, const uint32_t (&s)[4], const uint4& aux) {
    uint4 o = make_uint4(s[0], s[1], s[2], s[3]);
    if (MODE == kCtr || MODE == kCbcDec) {
        o.x ^= aux.x;
        o.y ^= aux.y;
        o.z ^= aux.z;
        o.w ^= aux.w;
    }
    __stcs(a.out + idx, o);
}

template <int MODE, int BPT>
__device__ __forceinline__ void load_tile(const EcbArgs& a, uint64_t t0b, uint32_t (&s)[BPT][4], uint4 (&aux)[BPT]) {
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const uint64_t idx = t0b + threadIdx.x + (uint64_t)b * blockDim.x;
        load_block<MODE>(a, idx, idx < a.nblocks, s[b], aux[b]);
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
    const uint64_t n = a.nblocks;
    const uint64_t tile = (uint64_t)blockDim.x * BPT;
    const uint64_t stride = (uint64_t)gridDim.x * tile;
    uint64_t t0b = (uint64_t)blockIdx.x * tile;
    uint32_t s[BPT][4];
    uint4 aux[BPT];  // CTR: data; CBC: previous ciphertext block
    // The first tile's loads go out before the table fill, so their memory
    // latency overlaps it (it dominates calls of a tile or two per CTA) --
    // except where holding 4 states and their mode data across the fill would
    // spill registers.
    constexpr bool kEarly = !(BPT == 4 && (MODE == kCtr || MODE == kCbcDec));
    if (kEarly) load_tile<MODE, BPT>(a, t0b, s, aux);
    fill_tables(A, DECRYPT);
    __syncthreads();
    if (!kEarly) load_tile<MODE, BPT>(a, t0b, s, aux);

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t L0 = A | (lane << 2);
    const uint32_t L1 = L0 | 128u;
    // Only the last tile is partial: a thread leaves once its next block is past the end.
    while (t0b + threadIdx.x < n) {
        cipher<NR, DECRYPT, BPT>(s, ParamKeys{a.rk}, L0, L1);
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const uint64_t idx = t0b + threadIdx.x + (uint64_t)b * blockDim.x;
            if (idx < n) store_block<MODE>(a, idx, s[b], aux[b]);
        }
        t0b += stride;
        if (t0b + threadIdx.x >= n) break;
        load_tile<MODE, BPT>(a, t0b, s, aux);
    }
}

// ------------------------------------------------------------ compact tables
//
// Calls too small to fill the GPU are bound by latency, not by the lookup rate:
// the 32x replicated tables (128-160 KiB per CTA) would take longer to write
// than the few blocks each CTA enciphers.  This variant keeps each of T0..T3
// (and the inverse S-box) once, 4-5 KiB of shared memory: one word per thread
// to write.  Its lookups may meet bank conflicts (32 lanes, random bytes, one
// copy), which costs little when every warp is one of a handful on its SM.
// Word x of table k sits at byte 1024*k + 4*x; the inverse S-box (its value in
// all four bytes) follows at 4096.

constexpr uint32_t kCompactWords = 5 * 256;

// AES_KERNEL_TABLE takes the compact tables up to this many blocks per SM
// (measured crossover on the GB300: below it the replicated tables' fill costs
// more than the compact tables' bank conflicts).
constexpr uint64_t kCompactBlocksPerSm = 128;

template <int K>
__device__ __forceinline__ uint32_t byte4(uint32_t w) {  // 4 * (byte K of w)
    return __byte_perm(w, 0u, 0x4440u | K) << 2;
}

__device__ __forceinline__ void fill_compact(uint32_t T, bool decrypt) {
    const uint32_t* t0 = decrypt ? g_tab.td0 : g_tab.te0;
    for (uint32_t x = threadIdx.x; x < 256u; x += blockDim.x) {
        const uint32_t v = __ldg(t0 + x);
        const uint32_t si = decrypt ? __ldg(g_tab.si4 + x) : 0u;
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) sts(T + 1024u * k + 4u * x, __funnelshift_l(v, v, 8u * k));
        if (decrypt) sts(T + 4096u + 4u * x, si);
    }
}

__device__ __forceinline__ void enc_round_c(uint32_t (&s)[4], uint32_t T, uint4 k) {
    uint32_t t[4];
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
        t[j] = lds(T + byte4<0>(s[j])) ^ lds_off<1024>(T + byte4<1>(s[(j + 1) & 3])) ^
               lds_off<2048>(T + byte4<2>(s[(j + 2) & 3])) ^ lds_off<3072>(T + byte4<3>(s[(j + 3) & 3])) ^ kk[j];
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// S[x] is byte 0 of T2[x], byte 1 of T3[x], byte 2 of T0[x], byte 3 of T1[x].
__device__ __forceinline__ void enc_last_c(uint32_t (&s)[4], uint32_t T, uint4 k) {
    uint32_t t[4];
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t o = merge(lds_off<2048>(T + byte4<0>(s[j])), lds_off<3072>(T + byte4<1>(s[(j + 1) & 3])), 0xffu);
        o = merge(o, lds(T + byte4<2>(s[(j + 2) & 3])), 0xffffu);
        o = merge(o, lds_off<1024>(T + byte4<3>(s[(j + 3) & 3])), 0xffffffu);
        t[j] = o ^ kk[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

__device__ __forceinline__ void dec_round_c(uint32_t (&s)[4], uint32_t T, uint4 k) {
    uint32_t t[4];
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
        t[j] = lds(T + byte4<0>(s[j])) ^ lds_off<1024>(T + byte4<1>(s[(j + 3) & 3])) ^
               lds_off<2048>(T + byte4<2>(s[(j + 2) & 3])) ^ lds_off<3072>(T + byte4<3>(s[(j + 1) & 3])) ^ kk[j];
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

__device__ __forceinline__ void dec_last_c(uint32_t (&s)[4], uint32_t T, uint4 k) {
    uint32_t t[4];
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t o = merge(lds_off<4096>(T + byte4<0>(s[j])), lds_off<4096>(T + byte4<1>(s[(j + 3) & 3])), 0xffu);
        o = merge(o, lds_off<4096>(T + byte4<2>(s[(j + 2) & 3])), 0xffffu);
        o = merge(o, lds_off<4096>(T + byte4<3>(s[(j + 1) & 3])), 0xffffffu);
        t[j] = o ^ kk[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

template <int NR, bool DECRYPT>
__device__ __forceinline__ void cipher_compact(uint32_t (&s)[4], const ParamKeys& ks, uint32_t T) {
    const uint4 k0 = ks.get(0);
    s[0] ^= k0.x;
    s[1] ^= k0.y;
    s[2] ^= k0.z;
    s[3] ^= k0.w;
#pragma unroll
    for (int r = 1; r < NR; ++r) {
        if (DECRYPT)
            dec_round_c(s, T, ks.get(r));
        else
            enc_round_c(s, T, ks.get(r));
    }
    if (DECRYPT)
        dec_last_c(s, T, ks.get(NR));
    else
        enc_last_c(s, T, ks.get(NR));
}

// One block per thread, grid-stride; the first block's load goes out before the fill.
template <int NR, int MODE>
__global__ void __launch_bounds__(256) table_compact_kernel(const EcbArgs a) {
    constexpr bool DECRYPT = (MODE == kDec || MODE == kCbcDec);
    __shared__ __align__(16) uint32_t tab[kCompactWords];
    const uint64_t n = a.nblocks;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t s[4];
    uint4 aux;
    load_block<MODE>(a, i, i < n, s, aux);
    const uint32_t T = smem_base(tab);
    fill_compact(T, DECRYPT);
    __syncthreads();
    while (i < n) {
        cipher_compact<NR, DECRYPT>(s, ParamKeys{a.rk}, T);
        store_block<MODE>(a, i, s, aux);
        i += stride;
        if (i >= n) break;
        load_block<MODE>(a, i, true, s, aux);
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
        case 0: return table_compact_kernel<NR, MODE>;
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

// bpt 0 selects the compact-table kernel.
KernelFn pick(int nr, int mode, int bpt) {
    switch (nr) {
        case 10: return pick_mode<10>(mode, bpt);
        case 12: return pick_mode<12>(mode, bpt);
        case 14: return pick_mode<14>(mode, bpt);
        default: return nullptr;
    }
}

}  // namespace

uint64_t compact_limit_blocks(int sms) { return (uint64_t)sms * kCompactBlocksPerSm; }

int launch_table(const EcbArgs& a, int nr, Mode mode, int threads, int bpt, int variant, cudaStream_t stream) {
    DeviceInfo info;
    int rc = current_device_info(&info);
    if (rc) return rc;
    const uint64_t n = a.nblocks;
    const uint64_t sms = (uint64_t)info.sms;
    if (variant == AES_KERNEL_TABLE) variant = n <= compact_limit_blocks(info.sms) ? AES_KERNEL_TABLE_COMPACT
                                                                                   : AES_KERNEL_TABLE_REPLICATED;
    KernelFn fn = pick(nr, mode, variant == AES_KERNEL_TABLE_COMPACT ? 0 : bpt);
    if (!fn) return fail(AES_ERR_ARG, "no table kernel for nr=%d mode=%d blocks_per_thread=%d", nr, (int)mode, bpt);
    unsigned grid;
    int smem = 0;
    if (variant == AES_KERNEL_TABLE_COMPACT) {
        // A warp per 32 blocks, spread over the SMs (at most 8 warps per CTA, 8 CTAs per SM).
        const uint64_t warps = (n + 31) / 32;
        uint64_t per_cta = (warps + sms - 1) / sms;
        if (per_cta > 8) per_cta = 8;
        const uint64_t ctas = (warps + per_cta - 1) / per_cta;
        grid = (unsigned)(ctas < 8 * sms ? ctas : 8 * sms);
        threads = (int)(32 * per_cta);
    } else {
        // Dynamic shared memory: the whole opt-in limit, so the 64 KiB-aligned
        // layout fits wherever the dynamic window starts (the kernel re-checks).
        smem = info.smem_optin;
        rc = set_max_dynamic_smem((const void*)fn, smem);
        if (rc) return rc;
        // One CTA per SM.  When each CTA takes only a few tiles, shrink the CTA so
        // the SMs share the blocks evenly: `iters` tiles each at the given shape
        // become `iters` tiles of just enough threads to cover n.
        const uint64_t per_cta = (uint64_t)threads * (uint64_t)bpt;
        const uint64_t iters = (n + sms * per_cta - 1) / (sms * per_cta);
        if (iters <= 64) {
            uint64_t t = (n + sms * bpt * iters - 1) / (sms * bpt * iters);
            t = (t + 31) / 32 * 32;
            if (t < 64) t = 64;
            if (t < (uint64_t)threads) threads = (int)t;
        }
        const uint64_t tile = (uint64_t)threads * (uint64_t)bpt;
        const uint64_t want = (n + tile - 1) / tile;
        grid = (unsigned)(want < sms ? want : sms);
    }
    fn<<<grid, threads, smem, stream>>>(a);
    cudaError_t e = cudaGetLastError();
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
