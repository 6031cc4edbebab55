// The cipher with the round count known only at run time, and round keys
// staged in shared memory: used where several key sizes share one kernel and
// the round keys come from memory anyway (batch.cu, resident.cu).
#pragma once

#include "aes_rounds.cuh"

namespace gbaes {

// One compact loop body serves every key size.
template <bool DECRYPT, int BPT, class KS>
__device__ __forceinline__ void cipher_rt(uint32_t (&s)[BPT][4], const KS& ks, int nr, uint32_t L0, uint32_t L1) {
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
#pragma unroll 1
    for (int r = 1; r < nr; ++r) {
        const uint4 k = ks.get(r);
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            if (DECRYPT)
                dec_round(s[b], L0, L1, k);
            else
                enc_round(s[b], L0, L1, k);
        }
    }
    const uint4 k = ks.get(nr);
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        if (DECRYPT)
            dec_last(s[b], L0, k);
        else
            enc_last(s[b], L0, L1, k);
    }
}

// Round keys staged in a shared-memory slot (16 B per round).
struct SmemKeys {
    uint32_t slot;
    __device__ __forceinline__ uint4 get(int r) const {
        uint4 k;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(k.x), "=r"(k.y), "=r"(k.z), "=r"(k.w)
                     : "r"(slot + 16u * (uint32_t)r));
        return k;
    }
};

}  // namespace gbaes
