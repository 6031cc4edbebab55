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
//    again folded into the round keys.  Decryption runs on A^-1 of the state,
//    where the two A^-1 join InvMixColumns and each inverse S-box is F itself
//    (decrypt_half).
//  * ShiftRows is a renaming of planes (across the two halves of a split state,
//    see "half states" below); MixColumns, the decryption's column map and
//    AddRoundKey are XORs.
//
// The kernel runs F as a cover by three-input lookup tables and the column
// maps as generated XOR programs (sbox_lut3.h, one LOP3 each).  The circuit and
// those programs are checked at compile time against the S-box and the column
// maps of aes_tables.h (static_asserts below).  Everything here is plain C++
// usable on the host as well as on the device.
#pragma once

#include <cstdint>

#include "aes_tables.h"
#include "sbox_lut3.h"

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

// Three-input lookup table: bit i of imm is the result for operand bits (a, b, c) =
// (i >> 2 & 1, i >> 1 & 1, i & 1), applied to 32 bit positions at once.  Lop3Eval
// evaluates it with plain logic (usable in constant expressions); Lop3 issues
// PTX lop3 on the device, one LOP3 instruction.
struct Lop3Eval {
    GBAES_HD constexpr uint32_t operator()(uint32_t a, uint32_t b, uint32_t c, uint32_t imm) const {
        uint32_t r = 0;
        for (uint32_t i = 0; i < 8; ++i)
            if ((imm >> i) & 1u) r |= ((i & 4u) ? a : ~a) & ((i & 2u) ? b : ~b) & ((i & 1u) ? c : ~c);
        return r;
    }
};
struct Lop3 {
#ifdef __CUDA_ARCH__
    template <class Imm>
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b, uint32_t c, Imm) const {
        uint32_t d;
        asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(Imm::value));
        return d;
    }
#else
    constexpr uint32_t operator()(uint32_t a, uint32_t b, uint32_t c, uint32_t imm) const {
        return Lop3Eval{}(a, b, c, imm);
    }
#endif
};

// S-box without its affine constant, then XOR with 8 key planes (k[t] for bit t),
// in place on one byte's 8 planes: the circuit mapped onto three-input tables
// (sbox_lut3.h), the key riding on its last tables.
GBAES_HD inline void sbox_planes_key(uint32_t* x, const uint32_t (&k)[8]) { sbox_key_lut3(x, k, Lop3{}); }

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

// The same, exhaustively, for the table-mapped network the kernel runs, with all-zero
// and all-one key planes: F(x) ^ key, F the S-box without its constant.
constexpr bool check_sbox_lut3() {
    for (int key = 0; key < 256; key += 255)
        for (int g = 0; g < 8; ++g) {
            uint32_t fwd[8] = {}, kp[8] = {};
            for (int t = 0; t < 8; ++t) {
                kp[t] = ((key >> t) & 1) ? 0xffffffffu : 0u;
                for (int k = 0; k < 32; ++k) fwd[t] |= (uint32_t)(((32 * g + k) >> t) & 1) << k;
            }
            sbox_key_lut3(fwd, kp, Lop3Eval{});
            for (int k = 0; k < 32; ++k) {
                int f = 0;
                for (int t = 0; t < 8; ++t) f |= (int)((fwd[t] >> k) & 1) << t;
                if ((f ^ 0x63 ^ key) != kAesTables.sbox[32 * g + k]) return false;
            }
        }
    return true;
}
static_assert(check_sbox_lut3(), "the table-mapped S-box network does not reproduce the S-box");

// A^-1 on one byte, straight from make_affine_inverse's rows.
constexpr uint8_t affine_inverse_byte(uint8_t v) {
    constexpr Rows8 M = make_affine_inverse();
    uint8_t r = 0;
    for (int i = 0; i < 8; ++i) {
        int p = 0;
        for (int j = 0; j < 8; ++j) p ^= ((M.r[i] >> j) & 1) & ((v >> j) & 1);
        r |= (uint8_t)(p << i);
    }
    return r;
}

// The linear programs against their maps written out with GF(2^8) products and
// A^-1, on all unit inputs at once (plane i holds unit vector i in bit i; the
// maps are linear, so the unit vectors decide them): MixColumns, the decryption
// column map A^-1 InvMixColumns A^-1 (A^-1 on each byte), and A^-1 on one byte.
constexpr bool check_linear_lut3() {
    constexpr uint8_t kMix[4] = {2, 3, 1, 1}, kInv[4] = {14, 11, 13, 9};
    uint32_t m[32] = {}, d[32] = {}, f[8] = {};
    for (int i = 0; i < 32; ++i) m[i] = d[i] = 1u << i;
    for (int i = 0; i < 8; ++i) f[i] = 1u << i;
    mix_column_lut3(m, Lop3Eval{});
    dec_mix_column_lut3(d, Lop3Eval{});
    affine_inv_byte_lut3(f, Lop3Eval{});
    for (int i = 0; i < 32; ++i) {
        uint8_t a[4] = {}, b[4] = {};
        a[i / 8] = (uint8_t)(1u << (i % 8));
        for (int q = 0; q < 4; ++q) b[q] = affine_inverse_byte(a[q]);
        for (int q = 0; q < 4; ++q) {
            uint8_t want_m = 0, inv_mix = 0;
            for (int j = 0; j < 4; ++j) {
                want_m ^= gf_mul_log(kMix[j], a[(q + j) & 3]);
                inv_mix ^= gf_mul_log(kInv[j], b[(q + j) & 3]);
            }
            const uint8_t want_d = affine_inverse_byte(inv_mix);
            for (int t = 0; t < 8; ++t) {
                if (((m[8 * q + t] >> i) & 1u) != ((want_m >> t) & 1u)) return false;
                if (((d[8 * q + t] >> i) & 1u) != ((want_d >> t) & 1u)) return false;
            }
        }
    }
    for (int i = 0; i < 8; ++i) {
        const uint8_t want = affine_inverse_byte((uint8_t)(1u << i));
        for (int t = 0; t < 8; ++t)
            if (((f[t] >> i) & 1u) != ((want >> t) & 1u)) return false;
    }
    return true;
}
static_assert(check_linear_lut3(), "the linear programs do not reproduce their maps");

// Byte permute: byte i of the result is byte (sel >> 4i) & 7 of the eight
// bytes {a (bytes 0-3), b (bytes 4-7)}; PRMT on the device.
GBAES_HD inline uint32_t byte_perm(uint32_t a, uint32_t b, uint32_t sel) {
#ifdef __CUDA_ARCH__
    return __byte_perm(a, b, sel);
#else
    const uint64_t x = ((uint64_t)b << 32) | a;
    uint32_t r = 0;
    for (int i = 0; i < 4; ++i) r |= (uint32_t)((x >> (8 * ((sel >> (4 * i)) & 7u))) & 0xffu) << (8 * i);
    return r;
#endif
}

// 32x32 bit transpose in place: afterwards bit r of w[c] = old bit c of w[r].
// Five exchange stages between words k and k+j (j = 16, 8, 4, 2, 1): word k
// keeps its bits under the mask and takes the partner's, shifted up by j, in
// the others; word k+j takes word k's, shifted down by j, under the mask.  The
// j = 16 and j = 8 stages move whole bytes, one byte permute per word.
GBAES_HD inline void transpose32(uint32_t* w) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t a = w[k], b = w[k + 16];
        w[k] = byte_perm(a, b, 0x5410u);       // a.lo16 | b.lo16 << 16
        w[k + 16] = byte_perm(a, b, 0x7632u);  // a.hi16 | b.hi16 << 16
    }
#pragma unroll
    for (int k = 0; k < 32; ++k)
        if ((k & 8) == 0) {
            const uint32_t a = w[k], b = w[k + 8];
            w[k] = byte_perm(a, b, 0x6240u);      // bytes a0 b0 a2 b2
            w[k + 8] = byte_perm(a, b, 0x7351u);  // bytes a1 b1 a3 b3
        }
    constexpr uint32_t kMask[3] = {0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 3; ++st) {
        const int j = 4 >> st;
        const uint32_t m = kMask[st], mh = m << j;
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if ((k & j) == 0) {
                const uint32_t a = w[k], b = w[k + j];
                w[k] = (a & ~mh) | ((b << j) & mh);
                w[k + j] = ((a >> j) & m) | (b & ~m);
            }
    }
}

// ------------------------------------------------------------- half states
//
// The kernel splits one 32-block state between a pair of lanes: half h (0 or 1)
// holds the 64 planes of state columns 2h and 2h+1.  Local byte l = 0..7 is
// state byte 8h + l (row l % 4 of column 2h + l / 4), its planes at
// s[8l .. 8l+7].  SubBytes, MixColumns and AddRoundKey stay inside a half;
// ShiftRows sends four of the eight bytes to the other half.  `other(v, p)`
// returns the other half's value of local plane p, v being this half's (on the
// device: a lane shuffle of v; in the CPU test harness: a read of the other
// thread's copy).

// ShiftRows, out(r, c) = in(r, c + r mod 4), on a half.  Row 0 (local bytes 0, 4)
// stays; in row 1 local byte 1 takes local byte 5 and byte 5 the other half's
// byte 1; row 2 (bytes 2, 6) comes from the other half's bytes 2, 6; in row 3
// byte 3 takes the other half's byte 7 and byte 7 takes local byte 3.  (The same
// rule holds for both halves, so one shuffle serves both.)
template <class Other>
GBAES_HD inline void shift_rows_half(uint32_t (&s)[64], const Other& other) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const uint32_t b1 = s[8 + t], b2 = s[16 + t], b3 = s[24 + t];
        const uint32_t b5 = s[40 + t], b6 = s[48 + t], b7 = s[56 + t];
        s[8 + t] = b5;
        s[40 + t] = other(b1, 8 + t);
        s[16 + t] = other(b2, 16 + t);
        s[48 + t] = other(b6, 48 + t);
        s[24 + t] = other(b7, 56 + t);
        s[56 + t] = b3;
    }
}

// InvShiftRows, out(r, c) = in(r, c - r mod 4), on a half: byte 1 takes the other
// half's byte 5, byte 5 takes local byte 1; bytes 2, 6 come from the other
// half's 2, 6; byte 3 takes local byte 7, byte 7 the other half's byte 3.
template <class Other>
GBAES_HD inline void inv_shift_rows_half(uint32_t (&s)[64], const Other& other) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const uint32_t b1 = s[8 + t], b2 = s[16 + t], b3 = s[24 + t];
        const uint32_t b5 = s[40 + t], b6 = s[48 + t], b7 = s[56 + t];
        s[8 + t] = other(b5, 40 + t);
        s[40 + t] = b1;
        s[16 + t] = other(b2, 16 + t);
        s[48 + t] = other(b6, 48 + t);
        s[24 + t] = b7;
        s[56 + t] = other(b3, 24 + t);
    }
}

// Key planes of one half: step r, local byte l at base[kKeyStepWords*r + 8l .. +7].
constexpr int kKeyHalfWords = 68;                 // 64 planes + 16 bytes, so the halves' rows use different banks
constexpr int kKeyStepWords = 2 * kKeyHalfWords;  // both halves of one step

struct HalfKeys {
    const uint32_t* base;  // this half's planes of step 0 (16-byte aligned)
    GBAES_HD void load8(int r, int l, uint32_t (&k)[8]) const {
        const uint32_t* q = base + kKeyStepWords * r + 8 * l;
#ifdef __CUDA_ARCH__
        const uint4 x = reinterpret_cast<const uint4*>(q)[0], y = reinterpret_cast<const uint4*>(q)[1];
        k[0] = x.x; k[1] = x.y; k[2] = x.z; k[3] = x.w;
        k[4] = y.x; k[5] = y.y; k[6] = y.z; k[7] = y.w;
#else
        for (int t = 0; t < 8; ++t) k[t] = q[t];
#endif
    }
};

template <class Keys>
GBAES_HD inline void add_key_half(uint32_t (&s)[64], const Keys& keys, int r) {
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        uint32_t k[8];
        keys.load8(r, l, k);
#pragma unroll
        for (int t = 0; t < 8; ++t) s[8 * l + t] ^= k[t];
    }
}

// MixColumns on the half's two columns (after ShiftRows and SubBytes), each as a
// generated program of two- and three-input XORs (sbox_lut3.h).  The round key
// was added before it, transformed (see make_key_planes).
GBAES_HD inline void mix_half(uint32_t (&s)[64]) {
    mix_column_lut3(&s[0], Lop3{});
    mix_column_lut3(&s[32], Lop3{});
}

// The decryption's column map A^-1 InvMixColumns A^-1 on the half's two columns
// (see decrypt_half), each as a generated XOR program.
GBAES_HD inline void dec_mix_half(uint32_t (&s)[64]) {
    dec_mix_column_lut3(&s[0], Lop3{});
    dec_mix_column_lut3(&s[32], Lop3{});
}

// A^-1 on each of the half's 8 bytes.
GBAES_HD inline void affine_inv_half(uint32_t (&s)[64]) {
#pragma unroll
    for (int l = 0; l < 8; ++l) affine_inv_byte_lut3(&s[8 * l], Lop3{});
}

// SubBytes with the key planes of step r added to its output, on a half.
template <class Keys>
GBAES_HD inline void sub_bytes_key_half(uint32_t (&s)[64], const Keys& keys, int r) {
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        uint32_t k[8];
        keys.load8(r, l, k);
        sbox_planes_key(&s[8 * l], k);
    }
}

// Encryption of a half state, with the key planes of make_key_planes: step 0
// before the first round, step r (the affine constant plus InvMixColumns of
// round key r, so that MixColumns turns it into round key r) on the S-box
// output of round r.  ShiftRows runs before SubBytes: the two commute, one
// moving whole bytes and the other mapping each byte.
template <int NR, class Keys, class Other>
GBAES_HD inline void encrypt_half(uint32_t (&s)[64], const Keys& keys, const Other& other) {
    add_key_half(s, keys, 0);
#pragma unroll 1
    for (int r = 1; r < NR; ++r) {
        shift_rows_half(s, other);
        sub_bytes_key_half(s, keys, r);
        mix_half(s);
    }
    shift_rows_half(s, other);
    sub_bytes_key_half(s, keys, NR);
}

// Straight inverse cipher on a half state, run on t = A^-1 s (A^-1 applied to
// every byte of the cipher state s).  The inverse S-box is A^-1 F(A^-1 x) for
// input x already carrying the affine constant (F the S-box without its
// constant), A^-1 is linear and commutes with InvShiftRows, so a round
//   s' = InvMixColumns(A^-1 F(A^-1 InvShiftRows(s)) ^ k)
// becomes, on t,
//   t' = A^-1 InvMixColumns A^-1 (F(InvShiftRows(t)) ^ A k):
// the encryption's S-box network with the key planes A k (make_key_planes),
// then one linear map per column.  The last round has no InvMixColumns: the
// output is A^-1 (F(InvShiftRows(t)) ^ A k).  The affine constant rides in the
// key planes as before.
template <int NR, class Keys, class Other>
GBAES_HD inline void decrypt_half(uint32_t (&s)[64], const Keys& keys, const Other& other) {
    add_key_half(s, keys, 0);
    affine_inv_half(s);
#pragma unroll 1
    for (int r = 1; r < NR; ++r) {
        inv_shift_rows_half(s, other);
        sub_bytes_key_half(s, keys, r);
        dec_mix_half(s);
    }
    inv_shift_rows_half(s, other);
    sub_bytes_key_half(s, keys, NR);
    affine_inv_half(s);
}

// InvMixColumns of one column word (byte q = row q): out_q = {0e}b_q + {0b}b_{q+1}
// + {0d}b_{q+2} + {09}b_{q+3}.
GBAES_HD constexpr uint8_t xtime8(uint8_t b) { return (uint8_t)((b << 1) ^ ((b & 0x80u) ? 0x1bu : 0u)); }
GBAES_HD constexpr uint32_t inv_mix_word(uint32_t w) {
    uint8_t b[4] = {}, o[4] = {};
    for (int q = 0; q < 4; ++q) b[q] = (uint8_t)(w >> (8 * q));
    for (int q = 0; q < 4; ++q) {
        const uint8_t x = b[q], y = b[(q + 1) & 3], z = b[(q + 2) & 3], v = b[(q + 3) & 3];
        const uint8_t x2 = xtime8(x), x4 = xtime8(x2), x8 = xtime8(x4);  // {0e} = 8 + 4 + 2
        const uint8_t y2 = xtime8(y), y8 = xtime8(xtime8(y2));          // {0b} = 8 + 2 + 1
        const uint8_t z4 = xtime8(xtime8(z)), z8 = xtime8(z4);          // {0d} = 8 + 4 + 1
        const uint8_t v8 = xtime8(xtime8(xtime8(v)));                   // {09} = 8 + 1
        o[q] = (uint8_t)(x8 ^ x4 ^ x2 ^ y8 ^ y2 ^ y ^ z8 ^ z4 ^ z ^ v8 ^ v);
    }
    return (uint32_t)o[0] | (uint32_t)o[1] << 8 | (uint32_t)o[2] << 16 | (uint32_t)o[3] << 24;
}

// The S-box's affine matrix A (without its constant) on each byte of a word:
// bit i of a byte becomes b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7}.
GBAES_HD constexpr uint32_t affine_word(uint32_t w) {
    uint32_t r = 0;
    for (int q = 0; q < 4; ++q) {
        const uint32_t b = (w >> (8 * q)) & 0xffu;
        for (int i = 0; i < 8; ++i) {
            const uint32_t bit = ((b >> i) ^ (b >> ((i + 4) & 7)) ^ (b >> ((i + 5) & 7)) ^ (b >> ((i + 6) & 7)) ^
                                  (b >> ((i + 7) & 7))) & 1u;
            r |= bit << (8 * q + i);
        }
    }
    return r;
}

// Key planes (0 or all ones) for each processing step, from a round-key
// schedule rk (4*(nr+1) words), plane p = 8*(state byte) + bit.
// Encryption: step 0 is rk[0]; step r (1 <= r < nr) is InvMixColumns(rk[r])
// XOR 0x63 in every byte, added to the S-box output before MixColumns
// (MixColumns is linear and maps 0x63 in all four bytes of a column to
// itself); step nr is rk[nr] XOR 0x63.  Decryption (straight inverse cipher
// on A^-1 of the state, see decrypt_half): step 0 is rk[nr] XOR 0x63; step r
// (r >= 1) is A applied to each byte of rk[nr - r], XORed with 0x63 first for
// r < nr.
GBAES_HD inline void make_key_planes(const uint32_t* rk, int nr, bool decrypt, uint32_t (*planes)[128]) {
    for (int r = 0; r <= nr; ++r) {
        const int src = decrypt ? nr - r : r;
        const bool fold = decrypt ? (r < nr) : (r >= 1);
        for (int p = 0; p < 128; ++p) {
            uint32_t w = rk[4 * src + p / 32];
            if (!decrypt && r >= 1 && r < nr) w = inv_mix_word(w);
            if (fold) w ^= 0x63636363u;
            if (decrypt && r >= 1) w = affine_word(w);
            planes[r][p] = ((w >> (p % 32)) & 1u) ? 0xffffffffu : 0u;
        }
    }
}

// Lays make_key_planes' output out for HalfKeys: step r, half h, local plane q
// at out[kKeyStepWords*r + kKeyHalfWords*h + q] (q = p - 64h).
GBAES_HD inline void split_key_planes(const uint32_t (*planes)[128], int nr, uint32_t* out) {
    for (int r = 0; r <= nr; ++r)
        for (int p = 0; p < 128; ++p) out[kKeyStepWords * r + kKeyHalfWords * (p / 64) + p % 64] = planes[r][p];
}

}  // namespace bs
}  // namespace gbaes
