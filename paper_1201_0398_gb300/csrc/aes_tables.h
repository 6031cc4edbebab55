// Compile-time AES tables for the GPU path (host and device).
//
// GF(2^8) arithmetic through exponent/logarithm tables of the generator {03}
// (modulus x^8+x^4+x^3+x+1, the field of Section 2.1), the S-box as the affine
// image of the multiplicative inverse, and the fused round tables of Eq. 1:
//
//   Te0[x] = bytes (02*S[x], S[x], S[x], 03*S[x])          (MixColumns column 0)
//   Td0[x] = bytes (0e*Si[x], 09*Si[x], 0d*Si[x], 0b*Si[x]) (InvMixColumns column 0)
//
// with "bytes (b0,b1,b2,b3)" meaning the little-endian 32-bit word b0 | b1<<8 |
// b2<<16 | b3<<24: byte k of a state word is row k of that column, the layout in
// which Section 3 reads a 16-byte block as four 32-bit values.  The other three
// tables of Eq. 1 are rotations: T_k[x] = rotl(T_0[x], 8k).
#pragma once

#include <cstdint>

namespace gbaes {

struct AesTables {
    uint8_t exp3[512];  // exp3[i] = {03}^i, doubled so exp3[log a + log b] needs no mod
    uint8_t log3[256];  // log3[{03}^i] = i; log3[0] unused
    uint8_t sbox[256];
    uint8_t inv_sbox[256];
    uint32_t te0[256];
    uint32_t td0[256];
    uint32_t si4[256];  // inverse S-box value replicated into all four bytes
};

constexpr uint8_t rotl8(uint8_t v, int n) { return (uint8_t)((v << n) | (v >> (8 - n))); }

constexpr AesTables make_aes_tables() {
    AesTables t{};
    // {03}^i: multiply by 03 = multiply by x (shift, reduce by 0x1b) plus identity.
    uint8_t e = 1;
    for (int i = 0; i < 255; ++i) {
        t.exp3[i] = e;
        t.exp3[i + 255] = e;
        t.log3[e] = (uint8_t)i;
        uint8_t twice = (uint8_t)((e << 1) ^ ((e & 0x80) ? 0x1b : 0));
        e = (uint8_t)(twice ^ e);
    }
    t.exp3[510] = t.exp3[0];
    t.exp3[511] = t.exp3[1];
    auto mul = [&t](uint8_t a, uint8_t b) -> uint8_t {
        return (a == 0 || b == 0) ? 0 : t.exp3[t.log3[a] + t.log3[b]];
    };
    for (int x = 0; x < 256; ++x) {
        uint8_t inv = x == 0 ? 0 : t.exp3[255 - t.log3[x]];
        uint8_t s = (uint8_t)(inv ^ rotl8(inv, 1) ^ rotl8(inv, 2) ^ rotl8(inv, 3) ^ rotl8(inv, 4) ^ 0x63);
        t.sbox[x] = s;
        t.inv_sbox[s] = (uint8_t)x;
    }
    for (int x = 0; x < 256; ++x) {
        uint8_t s = t.sbox[x];
        t.te0[x] = (uint32_t)mul(s, 2) | ((uint32_t)s << 8) | ((uint32_t)s << 16) | ((uint32_t)mul(s, 3) << 24);
        uint8_t si = t.inv_sbox[x];
        t.td0[x] = (uint32_t)mul(si, 0x0e) | ((uint32_t)mul(si, 0x09) << 8) | ((uint32_t)mul(si, 0x0d) << 16) |
                   ((uint32_t)mul(si, 0x0b) << 24);
        t.si4[x] = (uint32_t)si * 0x01010101u;
    }
    return t;
}

inline constexpr AesTables kAesTables = make_aes_tables();

// GF(2^8) product through the log tables.
constexpr uint8_t gf_mul_log(uint8_t a, uint8_t b) {
    return (a == 0 || b == 0) ? 0 : kAesTables.exp3[kAesTables.log3[a] + kAesTables.log3[b]];
}

}  // namespace gbaes
