// The cipher with the round count known only at run time, and round keys
// staged in shared memory: used where several key sizes share one kernel and
// the round keys come from memory anyway (batch.cu, resident.cu).
#pragma once

#include "aes_rounds.cuh"

namespace gbaes {

// One compact loop body serves every key size.  KS::get(r, b) is round r's key
// for state b; unless KS::kPerState, every state shares one key, loaded once
// per round.
template <bool DECRYPT, int BPT, class KS>
__device__ __forceinline__ void cipher_rt(uint32_t (&s)[BPT][4], const KS& ks, int nr, uint32_t L0, uint32_t L1) {
    constexpr int NK = KS::kPerState ? BPT : 1;
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const uint4 k = ks.get(0, b < NK ? b : 0);
        s[b][0] ^= k.x;
        s[b][1] ^= k.y;
        s[b][2] ^= k.z;
        s[b][3] ^= k.w;
    }
#pragma unroll 1
    for (int r = 1; r < nr; ++r) {
        uint4 k[NK];
#pragma unroll
        for (int b = 0; b < NK; ++b) k[b] = ks.get(r, b);
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            if (DECRYPT)
                dec_round(s[b], L0, L1, k[b < NK ? b : 0]);
            else
                enc_round(s[b], L0, L1, k[b < NK ? b : 0]);
        }
    }
    uint4 k[NK];
#pragma unroll
    for (int b = 0; b < NK; ++b) k[b] = ks.get(nr, b);
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        if (DECRYPT)
            dec_last(s[b], L0, k[b < NK ? b : 0]);
        else
            enc_last(s[b], L0, L1, k[b < NK ? b : 0]);
    }
}

// Round keys staged in a shared-memory slot (16 B per round), one key for every state.
struct SmemKeys {
    static constexpr bool kPerState = false;
    uint32_t slot;
    __device__ __forceinline__ uint4 get(int r, int) const { return get(r); }
    __device__ __forceinline__ uint4 get(int r) const {
        uint4 k;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(k.x), "=r"(k.y), "=r"(k.z), "=r"(k.w)
                     : "r"(slot + 16u * (uint32_t)r));
        return k;
    }
};

// One schedule in global memory (through L1) for every state.
struct OneGlobalKey {
    static constexpr bool kPerState = false;
    const uint4* p;
    __device__ __forceinline__ uint4 get(int r, int) const { return __ldg(p + r); }
};

// A schedule in global memory per state (states of different messages).
template <int BPT>
struct StateKeys {
    static constexpr bool kPerState = true;
    const uint4* const (&p)[BPT];
    __device__ __forceinline__ uint4 get(int r, int b) const { return __ldg(p[b] + r); }
};

}  // namespace gbaes
