// Bitsliced AES: the S-box as a Boolean circuit over bit planes.
//
// A "plane" is a 32-bit word holding one bit position of 32 different blocks
// (bit k of the plane = that bit of block k).  The 128 planes of a state are
// indexed p = 8*b + t for state byte b (0..15, byte 4c+r = row r of column c,
// Section 2.1's layout) and bit t of that byte.  Every AES step is then plain
// bitwise logic on planes, with no table lookups:
//
//  * SubBytes: the multiplicative inverse in GF(2^8) computed in the tower
//    field GF((2^4)^2).  A byte a = ah*Y + al with ah, al in GF(2^4) =
//    GF(2)[z]/(z^4+z+1) and Y^2 = Y + lambda has inverse
//        a^-1 = (ah * d^-1) Y + ((ah + al) * d^-1),  d = lambda*ah^2 + ah*al + al^2,
//    and d^-1 in GF(2^4) is four 4-input Boolean functions (3 LOP3 each, truth
//    tables computed at compile time).  The change of basis between
//    the AES field and the tower field is a linear map found at compile time
//    (make_tower below) and merged with the S-box's affine map.  The affine
//    constant 0x63 is not applied here: it passes unchanged through ShiftRows
//    and MixColumns (each MixColumns row sums to 1), so the caller XORs it into
//    the round keys instead.
//  * ShiftRows is a renaming of planes; MixColumns and AddRoundKey are XORs;
//    InvMixColumns is MixColumns after the preprocessing
//    a0 ^= 4(a0^a2), a2 ^= 4(a0^a2), a1 ^= 4(a1^a3), a3 ^= 4(a1^a3).
//
// The derivation is checked exhaustively at compile time against the S-box of
// aes_tables.h (static_asserts at the end of this file).  Everything here is
// plain C++ usable on the host as well as on the device.
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

constexpr uint8_t gf16_mul(uint8_t a, uint8_t b) {  // GF(2)[z]/(z^4+z+1)
    uint8_t p = 0;
    for (int i = 0; i < 4; ++i)
        if ((b >> i) & 1) p ^= (uint8_t)(a << i);
    for (int d = 6; d >= 4; --d)
        if ((p >> d) & 1) p ^= (uint8_t)(0x13 << (d - 4));
    return p & 15;
}

constexpr uint8_t gf16_inv(uint8_t a) {  // a^14
    uint8_t r = 1;
    for (int i = 0; i < 14; ++i) r = gf16_mul(r, a);
    return a ? r : 0;
}

constexpr uint8_t gf256_pow(uint8_t a, int e) {
    uint8_t r = 1;
    for (int i = 0; i < e; ++i) r = gf_mul_log(r, a);
    return r;
}

// Applies an 8x8 GF(2) matrix given as rows (bit j of row i = M[i][j]).
constexpr uint8_t apply8(const uint8_t (&rows)[8], uint8_t x) {
    uint8_t y = 0;
    for (int i = 0; i < 8; ++i) {
        uint8_t v = rows[i] & x, par = 0;
        for (int j = 0; j < 8; ++j) par ^= (v >> j) & 1;
        y |= (uint8_t)(par << i);
    }
    return y;
}

struct Tower {
    uint8_t lambda;         // Y^2 + Y + lambda irreducible over GF(16)
    uint8_t enc_in[8];      // AES byte -> tower (bits 0..3 = al, 4..7 = ah)
    uint8_t enc_out[8];     // tower -> AES byte, then the affine matrix (no constant)
    uint8_t dec_in[8];      // AES byte -> inverse affine matrix (no constant) -> tower
    uint8_t dec_out[8];     // tower -> AES byte
    bool ok;
};

// Inverts an 8x8 GF(2) matrix (rows); ok=false if singular.
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

// Rows of the matrix whose columns are the given bytes (column j = image of bit j).
constexpr void rows_from_columns(const uint8_t (&cols)[8], uint8_t (&rows)[8]) {
    for (int i = 0; i < 8; ++i) {
        uint8_t r = 0;
        for (int j = 0; j < 8; ++j) r |= (uint8_t)(((cols[j] >> i) & 1) << j);
        rows[i] = r;
    }
}

constexpr void mat_mul8(const uint8_t (&a)[8], const uint8_t (&b)[8], uint8_t (&c)[8]) {  // c = a * b
    uint8_t cols[8] = {};
    for (int j = 0; j < 8; ++j) cols[j] = apply8(a, apply8(b, (uint8_t)(1u << j)));
    rows_from_columns(cols, c);
}

constexpr Tower make_tower() {
    Tower T{};
    // omega: a root of z^4 + z + 1 in the AES field (generates the subfield GF(16)).
    uint8_t omega = 0;
    for (int x = 2; x < 256 && !omega; ++x)
        if ((gf256_pow((uint8_t)x, 4) ^ (uint8_t)x ^ 1) == 0) omega = (uint8_t)x;
    // lambda: smallest with Y^2 + Y + lambda irreducible over GF(16).
    for (int l = 1; l < 16 && !T.lambda; ++l) {
        bool root = false;
        for (int y = 0; y < 16; ++y)
            if ((gf16_mul((uint8_t)y, (uint8_t)y) ^ (uint8_t)y ^ (uint8_t)l) == 0) root = true;
        if (!root) T.lambda = (uint8_t)l;
    }
    uint8_t lam256 = 0;  // lambda written in the AES field: sum lambda_i omega^i
    for (int i = 0; i < 4; ++i)
        if ((T.lambda >> i) & 1) lam256 ^= gf256_pow(omega, i);
    uint8_t beta = 0;  // a root of Y^2 + Y + lambda in the AES field
    for (int x = 2; x < 256 && !beta; ++x)
        if ((gf_mul_log((uint8_t)x, (uint8_t)x) ^ (uint8_t)x ^ lam256) == 0) beta = (uint8_t)x;
    // tower bit j -> AES element: bits 0..3 are al (omega^j), bits 4..7 are ah (omega^(j-4) * beta)
    uint8_t cols[8] = {};
    for (int j = 0; j < 4; ++j) {
        cols[j] = gf256_pow(omega, j);
        cols[4 + j] = gf_mul_log(gf256_pow(omega, j), beta);
    }
    uint8_t to_aes[8] = {}, to_tower[8] = {};
    rows_from_columns(cols, to_aes);
    T.ok = omega && T.lambda && beta && invert8(to_aes, to_tower);
    // affine matrix A: b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7}
    uint8_t A[8] = {}, Ainv[8] = {};
    for (int i = 0; i < 8; ++i)
        A[i] = (uint8_t)((1u << i) | (1u << ((i + 4) & 7)) | (1u << ((i + 5) & 7)) | (1u << ((i + 6) & 7)) |
                         (1u << ((i + 7) & 7)));
    T.ok = T.ok && invert8(A, Ainv);
    for (int i = 0; i < 8; ++i) {
        T.enc_in[i] = to_tower[i];
        T.dec_out[i] = to_aes[i];
    }
    mat_mul8(A, to_aes, T.enc_out);
    mat_mul8(to_tower, Ainv, T.dec_in);
    return T;
}

inline constexpr Tower kTower = make_tower();

// Scalar model of the circuit (compile-time check only).
constexpr uint8_t tower_inverse(uint8_t t) {
    const uint8_t al = t & 15, ah = t >> 4;
    const uint8_t d = gf16_mul(kTower.lambda, gf16_mul(ah, ah)) ^ gf16_mul(ah, al) ^ gf16_mul(al, al);
    const uint8_t di = gf16_inv(d);
    return (uint8_t)((gf16_mul(ah, di) << 4) | gf16_mul(ah ^ al, di));
}

constexpr bool check_tower() {
    if (!kTower.ok) return false;
    for (int x = 0; x < 256; ++x) {
        if ((apply8(kTower.enc_out, tower_inverse(apply8(kTower.enc_in, (uint8_t)x))) ^ 0x63) != kAesTables.sbox[x])
            return false;
        if (apply8(kTower.dec_out, tower_inverse(apply8(kTower.dec_in, (uint8_t)(x ^ 0x63)))) !=
            kAesTables.inv_sbox[x])
            return false;
    }
    return true;
}
static_assert(check_tower(), "tower-field S-box circuit does not reproduce the S-box");

// ------------------------------------------------------------ plane circuits

// The four constant matrices, by value (device code sees only constants).
struct Rows8 {
    uint8_t r[8];
};
enum : int { kEncIn = 0, kEncOut = 1, kDecIn = 2, kDecOut = 3 };
constexpr Rows8 tower_rows(int which) {
    Rows8 m{};
    for (int i = 0; i < 8; ++i)
        m.r[i] = which == kEncIn ? kTower.enc_in[i]
                 : which == kEncOut ? kTower.enc_out[i]
                 : which == kDecIn ? kTower.dec_in[i]
                                   : kTower.dec_out[i];
    return m;
}

// y = M x over 8 planes, M constant (rows): only the XORs M selects survive.
template <int WHICH>
GBAES_HD inline void lin8(const uint32_t (&x)[8], uint32_t (&y)[8]) {
    constexpr Rows8 M = tower_rows(WHICH);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if ((M.r[i] >> j) & 1) acc ^= x[j];
        y[i] = acc;
    }
}

// GF(16) product of plane quadruples (polynomial basis, z^4 = z + 1).
GBAES_HD inline void mul16(const uint32_t* a, const uint32_t* b, uint32_t* c) {
    const uint32_t p0 = a[0] & b[0];
    const uint32_t p1 = (a[0] & b[1]) ^ (a[1] & b[0]);
    const uint32_t p2 = (a[0] & b[2]) ^ (a[1] & b[1]) ^ (a[2] & b[0]);
    const uint32_t p3 = (a[0] & b[3]) ^ (a[1] & b[2]) ^ (a[2] & b[1]) ^ (a[3] & b[0]);
    const uint32_t p4 = (a[1] & b[3]) ^ (a[2] & b[2]) ^ (a[3] & b[1]);
    const uint32_t p5 = (a[2] & b[3]) ^ (a[3] & b[2]);
    const uint32_t p6 = a[3] & b[3];
    c[0] = p0 ^ p4;
    c[1] = p1 ^ p4 ^ p5;
    c[2] = p2 ^ p5 ^ p6;
    c[3] = p3 ^ p6;
}

// a^2 in GF(16): (a0 + a1 z + a2 z^2 + a3 z^3)^2 = (a0^a2) + a2 z + (a1^a3) z^2 + a3 z^3.
GBAES_HD inline void sq16(const uint32_t* a, uint32_t* c) {
    c[0] = a[0] ^ a[2];
    c[1] = a[2];
    c[2] = a[1] ^ a[3];
    c[3] = a[3];
}

// Product with the constant lambda (bits select which shifted copies are added).
GBAES_HD inline void mul16_lambda(const uint32_t* a, uint32_t* c) {
    constexpr uint8_t lam = kTower.lambda;
    uint32_t l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) l[i] = ((lam >> i) & 1) ? 0xffffffffu : 0u;
    mul16(a, l, c);
}

// Three-input Boolean function given by its truth table LUT (bit (a<<2|b<<1|c)
// of LUT = f(a,b,c)), applied bitwise: one LOP3 on the device.
template <int LUT>
GBAES_HD inline uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
#else
    uint32_t d = 0;
    for (int k = 0; k < 8; ++k)
        if ((LUT >> k) & 1)
            d |= ((k & 4) ? a : ~a) & ((k & 2) ? b : ~b) & ((k & 1) ? c : ~c);
    return d;
#endif
}

// Truth table of output bit I of the GF(16) inverse restricted to input bit 3 = D3,
// as a function of input bits (0, 1, 2) in LOP3 operand order (a, b, c).
constexpr int inv16_lut(int I, int D3) {
    int lut = 0;
    for (int k = 0; k < 8; ++k) {
        const int d = ((k >> 2) & 1) | (((k >> 1) & 1) << 1) | ((k & 1) << 2) | (D3 << 3);
        lut |= ((gf16_inv((uint8_t)d) >> I) & 1) << k;
    }
    return lut;
}

// GF(16) inverse (0 -> 0) of a plane quadruple: each output bit is a
// four-input function, i.e. two three-input LOP3s selected by d[3] (0xCA:
// a ? b : c), 12 operations in all.
GBAES_HD inline void inv16(const uint32_t* d, uint32_t* o) {
#define GBAES_INV16_BIT(I)                                                   \
    {                                                                        \
        const uint32_t lo = lop3<inv16_lut(I, 0)>(d[0], d[1], d[2]);         \
        const uint32_t hi = lop3<inv16_lut(I, 1)>(d[0], d[1], d[2]);         \
        o[I] = lop3<0xCA>(d[3], hi, lo);                                     \
    }
    GBAES_INV16_BIT(0)
    GBAES_INV16_BIT(1)
    GBAES_INV16_BIT(2)
    GBAES_INV16_BIT(3)
#undef GBAES_INV16_BIT
}

// Inverse in GF(2^8) through the tower field, on tower coordinates t[0..7].
GBAES_HD inline void tower_inv(const uint32_t (&t)[8], uint32_t (&o)[8]) {
    const uint32_t* al = t;
    const uint32_t* ah = t + 4;
    uint32_t a2[4], la2[4], hl[4], l2[4], d[4];
    sq16(ah, a2);
    mul16_lambda(a2, la2);
    mul16(ah, al, hl);
    sq16(al, l2);
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = la2[i] ^ hl[i] ^ l2[i];
    uint32_t di[4];
    inv16(d, di);
    uint32_t s[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) s[i] = ah[i] ^ al[i];
    mul16(s, di, o);       // low half: (ah + al) d^-1
    mul16(ah, di, o + 4);  // high half: ah d^-1
}

// S-box without its affine constant, in place on one byte's 8 planes.
GBAES_HD inline void sbox_planes(uint32_t* x) {
    uint32_t in[8], t[8], o[8], y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) in[i] = x[i];
    lin8<kEncIn>(in, t);
    tower_inv(t, o);
    lin8<kEncOut>(o, y);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = y[i];
}

// Inverse S-box for input already XORed with the affine constant, in place.
GBAES_HD inline void inv_sbox_planes(uint32_t* x) {
    uint32_t in[8], t[8], o[8], y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) in[i] = x[i];
    lin8<kDecIn>(in, t);
    tower_inv(t, o);
    lin8<kDecOut>(o, y);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = y[i];
}

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
