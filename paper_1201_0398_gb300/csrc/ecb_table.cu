// T-table AES kernels for sm_103a: ECB encryption/decryption, CTR, CBC decryption.
//
// Each round is Eq. 1 of the paper: four output words, each the XOR of four
// 32-bit table lookups and a round-key word,
//     O_j = T0[I_{j,0}] ^ T1[I_{j+1,1}] ^ T2[I_{j+2,2}] ^ T3[I_{j+3,3}] ^ K_j
// (indices of I mod 4), and for the inverse cipher the same with Td tables and
// I_{j-k,k}.  The paper keeps the tables in a texture (Section 3); here they are
// in shared memory, laid out so that every lookup is bank-conflict free and
// its address costs one PRMT:
//
//   * Every table is replicated 32 times, lane l reading copy l, so lane l
//     always hits bank l whatever its index.
//   * Entries are 64 words apart: word (64*x + 32*slot + l) of a 64 KiB region
//     holds T_{2*region+slot}[x] for lane l.  The byte address is then
//     x<<8 | slot<<7 | l<<2, so one __byte_perm drops state byte k into address
//     byte 1 next to a per-lane constant (l<<2 | slot<<7 | region base) -- no
//     shift, mask or add.  Region 1 (T2, T3) is reached through the load's
//     immediate offset.
//   * The 128 KiB (encryption) / 160 KiB (decryption, plus a 32x replicated
//     inverse S-box for the last round) live in dynamic shared memory at a
//     64 KiB-aligned shared-window address, so the region base fits in the
//     address's upper half and the PRMT can carry it.
//
// One CTA per SM (the tables fill most of the SM's shared memory), persistent
// over the input in tiles of threads*BPT blocks, each block a coalesced 16-byte
// load and store.  Round keys come from the kernel parameters (constant bank).
#include <cstdio>

#include "aes_tables.h"
#include "gbaes_internal.h"

namespace gbaes {

__constant__ AesTables c_tab = make_aes_tables();

__device__ int g_status;  // nonzero: a kernel found its shared-memory layout did not fit

constexpr uint32_t kRegion = 0x10000u;                 // one 64 KiB region: two tables
constexpr uint32_t kEncBytes = 2 * kRegion;            // T0|T1, T2|T3
constexpr uint32_t kSiOffset = 2 * kRegion;            // decryption: inverse S-box
constexpr uint32_t kDecBytes = 2 * kRegion + 0x8000u;  // + 256 entries x 32 lanes x 4 B

__device__ __forceinline__ uint32_t lds(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

template <uint32_t OFF>
__device__ __forceinline__ uint32_t lds_off(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
    return v;
}

__device__ __forceinline__ void sts(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Address of T_{2*region+slot}[byte k of w] for this lane, region offset aside:
// byte 0 <- lane constant (l<<2 | slot<<7), byte 1 <- byte k of w,
// bytes 2,3 <- the 64 KiB-aligned base carried in the lane constant.
template <int K>
__device__ __forceinline__ uint32_t taddr(uint32_t w, uint32_t lane_const) {
    return __byte_perm(w, lane_const, 0x7604u | (K << 4));
}

// (a & m) | (b & ~m): bytes of a where m is set, of b elsewhere.
__device__ __forceinline__ uint32_t merge(uint32_t a, uint32_t b, uint32_t m) { return (a & m) | (b & ~m); }

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123u); }

// One inner encryption round (Eq. 1) on state s with round-key words k0..k3.
__device__ __forceinline__ void enc_round(uint32_t (&s)[4], uint32_t L0, uint32_t L1, uint32_t k0, uint32_t k1,
                                          uint32_t k2, uint32_t k3) {
    uint32_t t[4];
    const uint32_t kk[4] = {k0, k1, k2, k3};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t a0 = lds(taddr<0>(s[j], L0));                            // T0[I_{j,0}]
        uint32_t a1 = lds(taddr<1>(s[(j + 1) & 3], L1));                  // T1[I_{j+1,1}]
        uint32_t a2 = lds_off<kRegion>(taddr<2>(s[(j + 2) & 3], L0));     // T2[I_{j+2,2}]
        uint32_t a3 = lds_off<kRegion>(taddr<3>(s[(j + 3) & 3], L1));     // T3[I_{j+3,3}]
        t[j] = a0 ^ a1 ^ a2 ^ a3 ^ kk[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// Last encryption round: SubBytes + ShiftRows + AddRoundKey.  S[x] is a byte of
// each rotated table: byte 0 of T2, byte 1 of T3, byte 2 of T0, byte 3 of T1.
__device__ __forceinline__ void enc_last(uint32_t (&s)[4], uint32_t L0, uint32_t L1, uint32_t k0, uint32_t k1,
                                         uint32_t k2, uint32_t k3) {
    uint32_t t[4];
    const uint32_t kk[4] = {k0, k1, k2, k3};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t e0 = lds_off<kRegion>(taddr<0>(s[j], L0));           // T2: byte 0 = S
        uint32_t e1 = lds_off<kRegion>(taddr<1>(s[(j + 1) & 3], L1)); // T3: byte 1 = S
        uint32_t e2 = lds(taddr<2>(s[(j + 2) & 3], L0));              // T0: byte 2 = S
        uint32_t e3 = lds(taddr<3>(s[(j + 3) & 3], L1));              // T1: byte 3 = S
        uint32_t o = merge(e0, e1, 0x000000ffu);
        o = merge(o, e2, 0x0000ffffu);
        o = merge(o, e3, 0x00ffffffu);
        t[j] = o ^ kk[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// One inner round of the equivalent inverse cipher: Td tables, I_{j-k,k}.
__device__ __forceinline__ void dec_round(uint32_t (&s)[4], uint32_t L0, uint32_t L1, uint32_t k0, uint32_t k1,
                                          uint32_t k2, uint32_t k3) {
    uint32_t t[4];
    const uint32_t kk[4] = {k0, k1, k2, k3};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t a0 = lds(taddr<0>(s[j], L0));                         // Td0[I_{j,0}]
        uint32_t a1 = lds(taddr<1>(s[(j + 3) & 3], L1));               // Td1[I_{j-1,1}]
        uint32_t a2 = lds_off<kRegion>(taddr<2>(s[(j + 2) & 3], L0));  // Td2[I_{j-2,2}]
        uint32_t a3 = lds_off<kRegion>(taddr<3>(s[(j + 1) & 3], L1));  // Td3[I_{j-3,3}]
        t[j] = a0 ^ a1 ^ a2 ^ a3 ^ kk[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// Inverse S-box entry for byte K of w: 32x replicated table, stride 32 words.
template <int K>
__device__ __forceinline__ uint32_t si_lookup(uint32_t w, uint32_t L0) {
    uint32_t b = (w >> (8 * K)) & 0xffu;
    return lds_off<kSiOffset>((b << 7) | L0);
}

// Last round of the inverse cipher: InvShiftRows + InvSubBytes + AddRoundKey.
__device__ __forceinline__ void dec_last(uint32_t (&s)[4], uint32_t L0, uint32_t k0, uint32_t k1, uint32_t k2,
                                         uint32_t k3) {
    uint32_t t[4];
    const uint32_t kk[4] = {k0, k1, k2, k3};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t d0 = si_lookup<0>(s[j], L0);
        uint32_t d1 = si_lookup<1>(s[(j + 3) & 3], L0);
        uint32_t d2 = si_lookup<2>(s[(j + 2) & 3], L0);
        uint32_t d3 = si_lookup<3>(s[(j + 1) & 3], L0);
        uint32_t o = merge(d0, d1, 0x000000ffu);
        o = merge(o, d2, 0x0000ffffu);
        o = merge(o, d3, 0x00ffffffu);
        t[j] = o ^ kk[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// Full cipher on BPT independent states, rounds interleaved across the states.
template <int NR, bool DECRYPT, int BPT>
__device__ __forceinline__ void cipher(uint32_t (&s)[BPT][4], const EcbArgs& a, uint32_t L0, uint32_t L1) {
#pragma unroll
    for (int b = 0; b < BPT; ++b)
#pragma unroll
        for (int j = 0; j < 4; ++j) s[b][j] ^= a.rk[j];
#pragma unroll
    for (int r = 1; r < NR; ++r) {
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            if (DECRYPT)
                dec_round(s[b], L0, L1, a.rk[4 * r], a.rk[4 * r + 1], a.rk[4 * r + 2], a.rk[4 * r + 3]);
            else
                enc_round(s[b], L0, L1, a.rk[4 * r], a.rk[4 * r + 1], a.rk[4 * r + 2], a.rk[4 * r + 3]);
        }
    }
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        if (DECRYPT)
            dec_last(s[b], L0, a.rk[4 * NR], a.rk[4 * NR + 1], a.rk[4 * NR + 2], a.rk[4 * NR + 3]);
        else
            enc_last(s[b], L0, L1, a.rk[4 * NR], a.rk[4 * NR + 1], a.rk[4 * NR + 2], a.rk[4 * NR + 3]);
    }
}

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
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw);
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint32_t A = (base + (kRegion - 1)) & ~(kRegion - 1);
    if (A + kNeed > base + dyn) {  // same outcome in every thread of every CTA
        if (threadIdx.x == 0) atomicOr(&g_status, 1);
        return;
    }

    // Fill: region r, slot s, entry x, lane l at word 64x + 32s + l = rotl(T0[x], 8(2r+s)).
    const uint32_t* t0 = DECRYPT ? c_tab.td0 : c_tab.te0;
    for (uint32_t w = threadIdx.x; w < (kEncBytes >> 2); w += blockDim.x) {
        const uint32_t x = (w >> 6) & 255u;
        const uint32_t rot = 8u * (2u * (w >> 14) + ((w >> 5) & 1u));
        const uint32_t v = t0[x];
        sts(A + 4u * w, __funnelshift_l(v, v, rot));
    }
    if (DECRYPT) {
        for (uint32_t w = threadIdx.x; w < 8192u; w += blockDim.x) sts(A + kSiOffset + 4u * w, c_tab.si4[w >> 5]);
    }
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t L0 = A | (lane << 2);
    const uint32_t L1 = L0 | 128u;
    const uint64_t n = a.nblocks;
    const uint64_t tile = (uint64_t)blockDim.x * BPT;
    const uint64_t stride = (uint64_t)gridDim.x * tile;

    for (uint64_t t0b = (uint64_t)blockIdx.x * tile; t0b < n; t0b += stride) {
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
                if (ok) v = __ldcs(a.in + idx[b]);
                aux[b] = v;
            } else {
                if (ok) v = __ldcs(a.in + idx[b]);
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
        cipher<NR, DECRYPT, BPT>(s, a, L0, L1);
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
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    const uint64_t per_cta = (uint64_t)threads * (uint64_t)bpt;
    const uint64_t want = (a.nblocks + per_cta - 1) / per_cta;
    const unsigned grid = (unsigned)(want < (uint64_t)info.sms ? want : (uint64_t)info.sms);
    fn<<<grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "table kernel launch: %s", cudaGetErrorString(e));
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
