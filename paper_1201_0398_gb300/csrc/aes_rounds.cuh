// Device-side AES rounds in the T-table form of Eq. 1, shared by the block
// kernels (ecb_table.cu) and the batched kernel (batch.cu).
//
// Shared-memory layout (bank-conflict free, one PRMT per lookup address):
//   * Every table is replicated 32 times; lane l reads copy l, so lane l always
//     hits bank l whatever byte it looks up.
//   * Region r (64 KiB) holds T_{2r} and T_{2r+1}: word 64*x + 32*slot + l is
//     T_{2r+slot}[x] for lane l, i.e. byte address x<<8 | slot<<7 | l<<2.  A
//     __byte_perm drops state byte k into address byte 1 beside a per-lane
//     constant (l<<2 | slot<<7 | the region base, which is 64 KiB aligned).
//     Region 1 is reached through the load's immediate offset.
//   * The inverse cipher adds the inverse S-box for its last round (32x
//     replicated, 32 words per entry) after the two regions.
// T_k[x] = rotl(T_0[x], 8k) (Eq. 1's four tables are rotations of one).
#pragma once

#include <cstdint>

#include "aes_tables.h"
#include "gbaes_internal.h"

namespace gbaes {

// Source of the shared-memory fills, read through the read-only global path.
static __device__ AesTables g_tab = make_aes_tables();

constexpr uint32_t kRegion = 0x10000u;                 // one 64 KiB region: two tables
constexpr uint32_t kEncBytes = 2 * kRegion;            // T0|T1, T2|T3
constexpr uint32_t kSiOffset = 2 * kRegion;            // inverse cipher: inverse S-box
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

// Streaming 16-byte global load that does not allocate in L1: the input is read
// once, and keeping it out of L1 keeps its fills out of the SRAM the
// shared-memory tables live in.
__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t smem_base(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    return dyn;
}

// 64 KiB-aligned start of the table layout inside the dynamic window.
__device__ __forceinline__ uint32_t table_base(uint32_t base) { return (base + (kRegion - 1)) & ~(kRegion - 1); }

// Fill store: ordered before the tables' first use by the __syncthreads that
// follows every fill, so it needs no compiler memory clobber (which would keep
// the next entry's global load from being issued early).
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(addr), "r"(v));
}

// Writes the tables of one direction into shared memory at A; threads tid =
// 0..nt-1 take part (fill_tables: the whole CTA), and the caller synchronises
// them afterwards.  Pair p = (entry x = p/4, table k = p%4): its 32 lane copies
// are 128 contiguous bytes at region k/2, slot k%2, written as eight 16-byte
// stores in an order rotated by p, so the 8 threads of each quarter-warp hit 8
// different bank groups.  A thread loads the entries of up to four pairs before
// storing any, so small CTAs (many pairs per thread) overlap the global loads.
__device__ __forceinline__ void fill_tables_n(uint32_t A, bool decrypt, uint32_t tid, uint32_t nt) {
    const uint32_t* t0 = decrypt ? g_tab.td0 : g_tab.te0;
    for (uint32_t p0 = tid; p0 < 1024u; p0 += 4u * nt) {
        uint32_t v[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t p = p0 + u * nt;
            v[u] = p < 1024u ? __ldg(t0 + (p >> 2)) : 0u;
        }
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t p = p0 + u * nt;
            if (p < 1024u) {
                const uint32_t k = p & 3u;
                const uint32_t val = __funnelshift_l(v[u], v[u], 8u * k);  // T_k[x] = rotl(T_0[x], 8k)
                const uint32_t base = A + (k >> 1) * kRegion + (p >> 2) * 256u + (k & 1u) * 128u;
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) sts128(base + 16u * ((j + p) & 7u), val);
            }
        }
    }
    if (decrypt) {
        for (uint32_t x0 = tid; x0 < 256u; x0 += 4u * nt) {
            uint32_t v[4];
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u) {
                const uint32_t x = x0 + u * nt;
                v[u] = x < 256u ? __ldg(g_tab.si4 + x) : 0u;
            }
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u) {
                const uint32_t x = x0 + u * nt;
                if (x < 256u) {
                    const uint32_t base = A + kSiOffset + x * 128u;
#pragma unroll
                    for (uint32_t j = 0; j < 8; ++j) sts128(base + 16u * ((j + x) & 7u), v[u]);
                }
            }
        }
    }
}

__device__ __forceinline__ void fill_tables(uint32_t A, bool decrypt) { fill_tables_n(A, decrypt, threadIdx.x, blockDim.x); }

// Address of T_{2*region+slot}[byte K of w] for this lane (region offset aside):
// byte 0 <- lane constant (l<<2 | slot<<7), byte 1 <- byte K of w, bytes 2,3 <-
// the 64 KiB-aligned base carried in the lane constant.
template <int K>
__device__ __forceinline__ uint32_t taddr(uint32_t w, uint32_t lane_const) {
    return __byte_perm(w, lane_const, 0x7604u | (K << 4));
}

// (a & m) | (b & ~m): bytes of a where m is set, of b elsewhere.
__device__ __forceinline__ uint32_t merge(uint32_t a, uint32_t b, uint32_t m) { return (a & m) | (b & ~m); }

// One inner encryption round (Eq. 1).
__device__ __forceinline__ void enc_round(uint32_t (&s)[4], uint32_t L0, uint32_t L1, uint4 k) {
    uint32_t t[4];
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t a0 = lds(taddr<0>(s[j], L0));                         // T0[I_{j,0}]
        uint32_t a1 = lds(taddr<1>(s[(j + 1) & 3], L1));               // T1[I_{j+1,1}]
        uint32_t a2 = lds_off<kRegion>(taddr<2>(s[(j + 2) & 3], L0));  // T2[I_{j+2,2}]
        uint32_t a3 = lds_off<kRegion>(taddr<3>(s[(j + 3) & 3], L1));  // T3[I_{j+3,3}]
        t[j] = a0 ^ a1 ^ a2 ^ a3 ^ kk[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// Last encryption round: SubBytes + ShiftRows + AddRoundKey.  S[x] is a byte of
// each rotated table: byte 0 of T2, byte 1 of T3, byte 2 of T0, byte 3 of T1.
__device__ __forceinline__ void enc_last(uint32_t (&s)[4], uint32_t L0, uint32_t L1, uint4 k) {
    uint32_t t[4];
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t e0 = lds_off<kRegion>(taddr<0>(s[j], L0));            // T2: byte 0 = S
        uint32_t e1 = lds_off<kRegion>(taddr<1>(s[(j + 1) & 3], L1));  // T3: byte 1 = S
        uint32_t e2 = lds(taddr<2>(s[(j + 2) & 3], L0));               // T0: byte 2 = S
        uint32_t e3 = lds(taddr<3>(s[(j + 3) & 3], L1));               // T1: byte 3 = S
        uint32_t o = merge(e0, e1, 0x000000ffu);
        o = merge(o, e2, 0x0000ffffu);
        o = merge(o, e3, 0x00ffffffu);
        t[j] = o ^ kk[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = t[j];
}

// One inner round of the equivalent inverse cipher: Td tables, I_{j-k,k}.
__device__ __forceinline__ void dec_round(uint32_t (&s)[4], uint32_t L0, uint32_t L1, uint4 k) {
    uint32_t t[4];
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
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

// Inverse S-box entry for byte K of w: 32x replicated table, 32 words per entry.
template <int K>
__device__ __forceinline__ uint32_t si_lookup(uint32_t w, uint32_t L0) {
    uint32_t b = (w >> (8 * K)) & 0xffu;
    return lds_off<kSiOffset>((b << 7) | L0);
}

// Last round of the inverse cipher: InvShiftRows + InvSubBytes + AddRoundKey.
__device__ __forceinline__ void dec_last(uint32_t (&s)[4], uint32_t L0, uint4 k) {
    uint32_t t[4];
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
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

// Round keys from the kernel parameters (uniform constant-bank operands).
struct ParamKeys {
    const uint32_t (&rk)[60];
    __device__ __forceinline__ uint4 get(int r) const {
        return make_uint4(rk[4 * r], rk[4 * r + 1], rk[4 * r + 2], rk[4 * r + 3]);
    }
};

// Full cipher on BPT independent states sharing one schedule, rounds
// interleaved across the states.
template <int NR, bool DECRYPT, int BPT, class KS>
__device__ __forceinline__ void cipher(uint32_t (&s)[BPT][4], const KS& ks, uint32_t L0, uint32_t L1) {
    {
        const uint4 k = ks.get(0);
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            s[b][0] ^= k.x;
            s[b][1] ^= k.y;
            s[b][2] ^= k.z;
            s[b][3] ^= k.w;
        }
    }
#pragma unroll
    for (int r = 1; r < NR; ++r) {
        const uint4 k = ks.get(r);
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            if (DECRYPT)
                dec_round(s[b], L0, L1, k);
            else
                enc_round(s[b], L0, L1, k);
        }
    }
    const uint4 k = ks.get(NR);
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        if (DECRYPT)
            dec_last(s[b], L0, k);
        else
            enc_last(s[b], L0, L1, k);
    }
}

}  // namespace gbaes
