// Bitsliced AES: the S-box as a Boolean circuit over bit planes.
//
// A "plane" is a 32-bit word holding one bit position of 32 different blocks
// (bit k of the plane = that bit of block k).  The 128 planes of a state are
// indexed p = 8*b + t for state byte b (0..15, byte 4c+r = row r of column c,
// Section 2.1's layout) and bit t of that byte.  Every AES step is then plain
// bitwise logic on planes, with no table lookups:
//
//  * SubBytes: the depth-16 S-box circuit of J. Boyar and R. Peralta ("A
//    depth-16 circuit for the AES S-box", 2012): a linear layer of XORs into 27
//    intermediate sums, a shared nonlinear middle of ANDs and XORs (the inverse
//    in a tower of subfields, 34 ANDs as written here) and a bottom linear layer
//    that also applies the S-box's affine map.  The affine constant 0x63 (the
//    circuit's XNORs) is not applied here: it passes unchanged through
//    ShiftRows and MixColumns (each MixColumns row sums to 1), so the caller
//    XORs it into the round keys instead.
//  * The inverse S-box reuses the same circuit: with F(z) = A inv(z) (the
//    circuit without the constant, A the affine matrix), the inverse S-box of
//    y is inv(A^-1 (y ^ 0x63)) = A^-1 F(A^-1 (y ^ 0x63)), the XOR with 0x63
//    again folded into the round keys; A^-1 costs one three-input XOR per bit.
//  * ShiftRows is a renaming of planes; MixColumns and AddRoundKey are XORs;
//    InvMixColumns is MixColumns after the preprocessing
//    a0 ^= 4(a0^a2), a2 ^= 4(a0^a2), a1 ^= 4(a1^a3), a3 ^= 4(a1^a3).
//
// The circuit is checked exhaustively at compile time against the S-box of
// aes_tables.h (static_asserts below).  Everything here is plain C++ usable on
// the host as well as on the device.
#pragma once

#include <cstdint>

#include "aes_tables.h"

#ifndef __CUDACC__
#define GBAES_HD
#else
#define GBAES_HD __host__ __device__
#endif

namespace gbaes {
namespace bs {

// ---------------------------------------------------------- scalar helpers

// Inverts an 8x8 GF(2) matrix (rows: bit j of row i = M[i][j]); false if singular.
constexpr bool invert8(const uint8_t (&m)[8], uint8_t (&inv)[8]) {
    uint8_t a[8] = {}, b[8] = {};
    for (int i = 0; i < 8; ++i) {
        a[i] = m[i];
        b[i] = (uint8_t)(1u << i);
    }
    for (int col = 0; col < 8; ++col) {
        int piv = -1;
        for (int r = col; r < 8; ++r)
            if ((a[r] >> col) & 1) {
                piv = r;
                break;
            }
        if (piv < 0) return false;
        uint8_t t = a[col]; a[col] = a[piv]; a[piv] = t;
        t = b[col]; b[col] = b[piv]; b[piv] = t;
        for (int r = 0; r < 8; ++r)
            if (r != col && ((a[r] >> col) & 1)) {
                a[r] ^= a[col];
                b[r] ^= b[col];
            }
    }
    for (int i = 0; i < 8; ++i) inv[i] = b[i];
    return true;
}

struct Rows8 {
    uint8_t r[8];
    bool ok;
};

// The inverse of the S-box's affine matrix A (b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7}).
constexpr Rows8 make_affine_inverse() {
    uint8_t A[8] = {}, Ainv[8] = {};
    for (int i = 0; i < 8; ++i)
        A[i] = (uint8_t)((1u << i) | (1u << ((i + 4) & 7)) | (1u << ((i + 5) & 7)) | (1u << ((i + 6) & 7)) |
                         (1u << ((i + 7) & 7)));
    Rows8 m{};
    m.ok = invert8(A, Ainv);
    for (int i = 0; i < 8; ++i) m.r[i] = Ainv[i];
    return m;
}

// ------------------------------------------------------------ plane circuits

// The S-box circuit without its affine constant: s = A inv(u) on planes, with
// u[i], s[i] = bit 7 - i of the input and output bytes (i = 0: the most
// significant bit), the bit order the published circuit is written in.
GBAES_HD constexpr void sbox_circuit(const uint32_t (&u)[8], uint32_t (&s)[8]) {
    // top linear layer
    const uint32_t t1 = u[0] ^ u[3], t2 = u[0] ^ u[5], t3 = u[0] ^ u[6], t4 = u[3] ^ u[5], t5 = u[4] ^ u[6];
    const uint32_t t6 = t1 ^ t5, t7 = u[1] ^ u[2], t8 = u[7] ^ t6, t9 = u[7] ^ t7, t10 = t6 ^ t7;
    const uint32_t t11 = u[1] ^ u[5], t12 = u[2] ^ u[5], t13 = t3 ^ t4, t14 = t6 ^ t11, t15 = t5 ^ t11;
    const uint32_t t16 = t5 ^ t12, t17 = t9 ^ t16, t18 = u[3] ^ u[7], t19 = t7 ^ t18, t20 = t1 ^ t19;
    const uint32_t t21 = u[6] ^ u[7], t22 = t7 ^ t21, t23 = t2 ^ t22, t24 = t2 ^ t10, t25 = t20 ^ t17;
    const uint32_t t26 = t3 ^ t16, t27 = t1 ^ t12;
    // nonlinear middle
    const uint32_t m1 = t13 & t6, m2 = t23 & t8, m3 = t14 ^ m1, m4 = t19 & u[7], m5 = m4 ^ m1;
    const uint32_t m6 = t3 & t16, m7 = t22 & t9, m8 = t26 ^ m6, m9 = t20 & t17, m10 = m9 ^ m6;
    const uint32_t m11 = t1 & t15, m12 = t4 & t27, m13 = m12 ^ m11, m14 = t2 & t10, m15 = m14 ^ m11;
    const uint32_t m16 = m3 ^ m2, m17 = m5 ^ t24, m18 = m8 ^ m7, m19 = m10 ^ m15, m20 = m16 ^ m13;
    const uint32_t m21 = m17 ^ m15, m22 = m18 ^ m13, m23 = m19 ^ t25, m24 = m22 ^ m23, m25 = m22 & m20;
    const uint32_t m26 = m21 ^ m25, m27 = m20 ^ m21, m28 = m23 ^ m25, m29 = m28 & m27, m30 = m26 & m24;
    const uint32_t m31 = m20 & m23, m32 = m27 ^ m25, m33 = m27 & m31, m34 = m24 ^ m25, m35 = m21 & m22;
    const uint32_t m36 = m24 & m35, m37 = m21 ^ m29, m38 = m32 ^ m33, m39 = m23 ^ m30, m40 = m34 ^ m36;
    const uint32_t m41 = m38 ^ m40, m42 = m37 ^ m39, m43 = m37 ^ m38, m44 = m39 ^ m40, m45 = m42 ^ m41;
    const uint32_t m46 = m44 & t6, m47 = m40 & t8, m48 = m39 & u[7], m49 = m43 & t16, m50 = m38 & t9;
    const uint32_t m51 = m37 & t17, m52 = m42 & t15, m53 = m45 & t27, m54 = m41 & t10, m55 = m44 & t13;
    const uint32_t m56 = m40 & t23, m57 = m39 & t19, m58 = m43 & t3, m59 = m38 & t22, m60 = m37 & t20;
    const uint32_t m61 = m42 & t1, m62 = m45 & t4, m63 = m41 & t2;
    // bottom linear layer (the affine map; its constant is left to the round keys)
    const uint32_t l0 = m61 ^ m62, l1 = m50 ^ m56, l2 = m46 ^ m48, l3 = m47 ^ m55, l4 = m54 ^ m58;
    const uint32_t l5 = m49 ^ m61, l6 = m62 ^ l5, l7 = m46 ^ l3, l8 = m51 ^ m59, l9 = m52 ^ m53;
    const uint32_t l10 = m53 ^ l4, l11 = m60 ^ l2, l12 = m48 ^ m51, l13 = m50 ^ l0, l14 = m52 ^ m61;
    const uint32_t l15 = m55 ^ l1, l16 = m56 ^ l0, l17 = m57 ^ l1, l18 = m58 ^ l8, l19 = m63 ^ l4;
    const uint32_t l20 = l0 ^ l1, l21 = l1 ^ l7, l22 = l3 ^ l12, l23 = l18 ^ l2, l24 = l15 ^ l9;
    const uint32_t l25 = l6 ^ l10, l26 = l7 ^ l9, l27 = l8 ^ l10, l28 = l11 ^ l14, l29 = l11 ^ l17;
    s[0] = l6 ^ l24;
    s[1] = l16 ^ l26;
    s[2] = l19 ^ l28;
    s[3] = l6 ^ l21;
    s[4] = l20 ^ l22;
    s[5] = l25 ^ l29;
    s[6] = l13 ^ l27;
    s[7] = l6 ^ l23;
}

// y = A^-1 x over 8 planes (x[t] = bit t): only the XORs the rows select survive.
GBAES_HD constexpr void affine_inverse_planes(const uint32_t (&x)[8], uint32_t (&y)[8]) {
    constexpr Rows8 M = make_affine_inverse();  // (a constant in device code too)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if ((M.r[i] >> j) & 1) acc ^= x[j];
        y[i] = acc;
    }
}

// S-box without its affine constant, in place on one byte's 8 planes (x[t] = bit t).
GBAES_HD constexpr void sbox_planes(uint32_t* x) {
    uint32_t u[8] = {}, o[8] = {};
#pragma unroll
    for (int i = 0; i < 8; ++i) u[i] = x[7 - i];
    sbox_circuit(u, o);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[7 - i] = o[i];
}

// Inverse S-box for input already XORed with the affine constant, in place:
// A^-1 F(A^-1 x), F the circuit.
GBAES_HD constexpr void inv_sbox_planes(uint32_t* x) {
    uint32_t in[8] = {}, z[8] = {}, u[8] = {}, o[8] = {}, f[8] = {}, y[8] = {};
#pragma unroll
    for (int i = 0; i < 8; ++i) in[i] = x[i];
    affine_inverse_planes(in, z);
#pragma unroll
    for (int i = 0; i < 8; ++i) u[i] = z[7 - i];
    sbox_circuit(u, o);
#pragma unroll
    for (int i = 0; i < 8; ++i) f[7 - i] = o[i];
    affine_inverse_planes(f, y);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = y[i];
}

// Exhaustive check: plane k of the input holds bit t of the byte value 32*g + k.
constexpr bool check_sbox_circuit() {
    if (!make_affine_inverse().ok) return false;
    for (int g = 0; g < 8; ++g) {
        uint32_t fwd[8] = {}, inv[8] = {};
        for (int t = 0; t < 8; ++t)
            for (int k = 0; k < 32; ++k) {
                const int x = 32 * g + k;
                fwd[t] |= (uint32_t)((x >> t) & 1) << k;
                inv[t] |= (uint32_t)(((x ^ 0x63) >> t) & 1) << k;
            }
        sbox_planes(fwd);
        inv_sbox_planes(inv);
        for (int k = 0; k < 32; ++k) {
            const int x = 32 * g + k;
            int f = 0, i = 0;
            for (int t = 0; t < 8; ++t) {
                f |= (int)((fwd[t] >> k) & 1) << t;
                i |= (int)((inv[t] >> k) & 1) << t;
            }
            if ((f ^ 0x63) != kAesTables.sbox[x] || i != kAesTables.inv_sbox[x]) return false;
        }
    }
    return true;
}
static_assert(check_sbox_circuit(), "the S-box circuit does not reproduce the S-box");

// Multiplication by {02} on one byte's planes (t[0] = least significant bit).
GBAES_HD inline void xtime_planes(const uint32_t* a, uint32_t* y) {
    y[0] = a[7];
    y[1] = a[0] ^ a[7];
    y[2] = a[1];
    y[3] = a[2] ^ a[7];
    y[4] = a[3] ^ a[7];
    y[5] = a[4];
    y[6] = a[5];
    y[7] = a[6];
}

// 32x32 bit transpose in place: afterwards bit r of w[c] = old bit c of w[r].
GBAES_HD inline void transpose32(uint32_t* w) {
    uint32_t m = 0x0000ffffu;
#pragma unroll
    for (int j = 16; j != 0; j >>= 1, m ^= (m << j)) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if ((k & j) == 0) {
                const uint32_t t = ((w[k] >> j) ^ w[k + j]) & m;
                w[k] ^= t << j;
                w[k + j] ^= t;
            }
        }
    }
}

// Planes of state byte b live at s[8b .. 8b+7].  key(p) returns the key plane
// (0 or all ones) of plane p for the round being applied.

// ShiftRows + MixColumns + AddRoundKey after SubBytes.  Output column c row r
// takes input byte 4((c+r)%4)+r (ShiftRows: row r rotated left by r).
template <class Key>
GBAES_HD inline void shift_mix_add(uint32_t (&s)[128], const Key& key) {
    uint32_t n[128];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint32_t* a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = &s[8 * (4 * ((c + r) & 3) + r)];
        // 2a_r + 3a_{r+1} + a_{r+2} + a_{r+3} = xtime(t_r) + t_{r+1} + a_{r+3},  t_r = a_r + a_{r+1}
        uint32_t tt[4][8];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < 8; ++t) tt[r][t] = a[r][t] ^ a[(r + 1) & 3][t];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint32_t x2[8];
            xtime_planes(tt[r], x2);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int p = 8 * (4 * c + r) + t;
                n[p] = x2[t] ^ tt[(r + 1) & 3][t] ^ a[(r + 3) & 3][t] ^ key(p);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < 128; ++p) s[p] = n[p];
}

// ShiftRows + AddRoundKey (last encryption round).
template <class Key>
GBAES_HD inline void shift_add(uint32_t (&s)[128], const Key& key) {
    uint32_t n[128];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int p = 8 * (4 * c + r) + t;
                n[p] = s[8 * (4 * ((c + r) & 3) + r) + t] ^ key(p);
            }
#pragma unroll
    for (int p = 0; p < 128; ++p) s[p] = n[p];
}

// InvShiftRows: output column c row r takes input byte 4((c-r)%4)+r.
GBAES_HD inline void inv_shift(uint32_t (&s)[128]) {
    uint32_t n[128];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < 8; ++t) n[8 * (4 * c + r) + t] = s[8 * (4 * ((c + 4 - r) & 3) + r) + t];
#pragma unroll
    for (int p = 0; p < 128; ++p) s[p] = n[p];
}

// AddRoundKey then InvMixColumns (as MixColumns after the {04} preprocessing).
template <class Key>
GBAES_HD inline void add_inv_mix(uint32_t (&s)[128], const Key& key) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t a[4][8];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < 8; ++t) a[r][t] = s[8 * (4 * c + r) + t] ^ key(8 * (4 * c + r) + t);
        uint32_t e[8], e2[8], u4[8], o[8], o2[8], v4[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            e[t] = a[0][t] ^ a[2][t];
            o[t] = a[1][t] ^ a[3][t];
        }
        xtime_planes(e, e2);
        xtime_planes(e2, u4);
        xtime_planes(o, o2);
        xtime_planes(o2, v4);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            a[0][t] ^= u4[t];
            a[2][t] ^= u4[t];
            a[1][t] ^= v4[t];
            a[3][t] ^= v4[t];
        }
        uint32_t tt[4][8];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < 8; ++t) tt[r][t] = a[r][t] ^ a[(r + 1) & 3][t];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint32_t x2[8];
            xtime_planes(tt[r], x2);
#pragma unroll
            for (int t = 0; t < 8; ++t) s[8 * (4 * c + r) + t] = x2[t] ^ tt[(r + 1) & 3][t] ^ a[(r + 3) & 3][t];
        }
    }
}

template <class Key>
GBAES_HD inline void add_key(uint32_t (&s)[128], const Key& key) {
#pragma unroll
    for (int p = 0; p < 128; ++p) s[p] ^= key(p);
}

// Encryption of the 32 blocks held as planes; keys(r) gives round r's key
// planes with the affine constant folded into rounds 1..nr.
template <int NR, class Keys>
GBAES_HD inline void encrypt_planes(uint32_t (&s)[128], const Keys& keys) {
    add_key(s, keys.round(0));
#pragma unroll 1
    for (int r = 1; r < NR; ++r) {
#pragma unroll
        for (int b = 0; b < 16; ++b) sbox_planes(&s[8 * b]);
        shift_mix_add(s, keys.round(r));
    }
#pragma unroll
    for (int b = 0; b < 16; ++b) sbox_planes(&s[8 * b]);
    shift_add(s, keys.round(NR));
}

// Straight inverse cipher; keys(r) gives the key planes applied at step r
// (r = 0: the last encryption round key, ...), constant folded as described.
template <int NR, class Keys>
GBAES_HD inline void decrypt_planes(uint32_t (&s)[128], const Keys& keys) {
    add_key(s, keys.round(0));
#pragma unroll 1
    for (int r = 1; r < NR; ++r) {
        inv_shift(s);
#pragma unroll
        for (int b = 0; b < 16; ++b) inv_sbox_planes(&s[8 * b]);
        add_inv_mix(s, keys.round(r));
    }
    inv_shift(s);
#pragma unroll
    for (int b = 0; b < 16; ++b) inv_sbox_planes(&s[8 * b]);
    add_key(s, keys.round(NR));
}

// Key planes (0 or all ones) for each processing step, from a round-key
// schedule rk (4*(nr+1) words).  Encryption: step r uses rk[r], XORed with
// 0x63 in every byte for r >= 1.  Decryption (straight inverse cipher): step r
// uses rk[nr - r], XORed with 0x63 in every byte for r < nr.
GBAES_HD inline void make_key_planes(const uint32_t* rk, int nr, bool decrypt, uint32_t (*planes)[128]) {
    for (int r = 0; r <= nr; ++r) {
        const int src = decrypt ? nr - r : r;
        const bool fold = decrypt ? (r < nr) : (r >= 1);
        for (int p = 0; p < 128; ++p) {
            const uint32_t w = rk[4 * src + p / 32] ^ (fold ? 0x63636363u : 0u);
            planes[r][p] = ((w >> (p % 32)) & 1u) ? 0xffffffffu : 0u;
        }
    }
}

// Round-key planes of one step, read by plane index.
struct StepKey {
    const uint32_t* k;
    GBAES_HD uint32_t operator()(int p) const { return k[p]; }
};

// All steps' key planes (e.g. in the kernel parameters).
struct PlaneKeys {
    const uint32_t (*planes)[128];
    GBAES_HD StepKey round(int r) const { return StepKey{planes[r]}; }
};

}  // namespace bs
}  // namespace gbaes
