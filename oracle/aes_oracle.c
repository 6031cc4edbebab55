/*
 * Plain CPU oracle for bulk AES (test infrastructure only).
 *
 * Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
 * bench.py load this file's library.  Nothing in the product path (the CUDA
 * library under paper_1201_0398_gb300/) includes, links or calls it, and it
 * shares no code, header, table or constant generator with that path.
 *
 * What it computes: the AES block cipher and its inverse exactly as the paper's
 * Section 2.1 describes it (128-bit blocks; 128/192/256-bit keys; 10/12/14
 * rounds; each round built from SubBytes, ShiftRows, MixColumns and
 * AddRoundKey over GF(2^8)), with the details Section 2.1 defers to its
 * reference [1], FIPS-197.  It is the plain, byte-oriented definition:
 *   - the S-box is the multiplicative inverse in GF(2^8) (modulus
 *     x^8+x^4+x^3+x+1) followed by the affine map, found by brute force;
 *   - MixColumns uses xtime; InvMixColumns uses a shift-and-add multiply;
 *   - the inverse cipher runs the steps in straight inverse order
 *     (Section 2.1: "all the steps ... performed in inverse order");
 *   - no T-tables (the fused form of Eq. 1 is what the GPU path does; the
 *     oracle deliberately does not).
 * Modes: ECB (Section 3), CTR (Section 3, counter = IV + block index, either
 * as one 128-bit big-endian integer or as the paper's four little-endian 32-bit
 * words with a carry chain x -> y -> z -> w), CBC decryption (Section 3, Eq. 2:
 * each block is XORed with the previous ciphertext block, the first with IV).
 *
 * State convention: state[r][c] = in[r + 4c] (FIPS-197 Section 3.4).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_KEYSIZE (-2)

/* ---------------------------------------------------------------- GF(2^8) */

/* xtime: multiplication by x (0x02) modulo x^8+x^4+x^3+x+1 (FIPS-197 4.2.1). */
static uint8_t xtime(uint8_t a) {
    return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0x00));
}

/* Product in GF(2^8) by repeated xtime and addition (FIPS-197 4.2). */
uint8_t oracle_gf_mul(uint8_t a, uint8_t b) {
    uint8_t acc = 0;
    while (b) {
        if (b & 1) acc ^= a;
        a = xtime(a);
        b >>= 1;
    }
    return acc;
}

/* Multiplicative inverse by exhaustive search; 0 maps to 0 (FIPS-197 5.1.1). */
static uint8_t gf_inverse(uint8_t a) {
    if (a == 0) return 0;
    for (int b = 1; b < 256; ++b)
        if (oracle_gf_mul(a, (uint8_t)b) == 1) return (uint8_t)b;
    return 0; /* unreachable: GF(2^8)* is a group */
}

static uint8_t SBOX[256];
static uint8_t INV_SBOX[256];
static pthread_once_t sbox_once = PTHREAD_ONCE_INIT;

/* S-box = affine transform of the inverse (FIPS-197 5.1.1, eq. 5.1):
 * b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i  (indices mod 8),
 * c = 0x63. */
static void build_sbox(void) {
    const uint8_t c = 0x63;
    for (int x = 0; x < 256; ++x) {
        uint8_t b = gf_inverse((uint8_t)x);
        uint8_t out = 0;
        for (int i = 0; i < 8; ++i) {
            int bit = ((b >> i) & 1) ^ ((b >> ((i + 4) % 8)) & 1) ^
                      ((b >> ((i + 5) % 8)) & 1) ^ ((b >> ((i + 6) % 8)) & 1) ^
                      ((b >> ((i + 7) % 8)) & 1) ^ ((c >> i) & 1);
            out |= (uint8_t)(bit << i);
        }
        SBOX[x] = out;
    }
    for (int x = 0; x < 256; ++x) INV_SBOX[SBOX[x]] = (uint8_t)x;
}

static void ensure_sbox(void) { pthread_once(&sbox_once, build_sbox); }

void oracle_sbox(uint8_t sbox[256], uint8_t inv_sbox[256]) {
    ensure_sbox();
    memcpy(sbox, SBOX, 256);
    memcpy(inv_sbox, INV_SBOX, 256);
}

/* ------------------------------------------------------------ key schedule */

static int rounds_for_bits(int bits) {
    switch (bits) {
        case 128: return 10;
        case 192: return 12;
        case 256: return 14;
        default: return -1;
    }
}

/* KeyExpansion (FIPS-197 5.2).  Words are 4-byte arrays w[i][0..3]; the
 * output holds 4*(Nr+1) words = 16*(Nr+1) bytes, word-major. */
int oracle_key_expansion(const uint8_t* key, int bits, uint8_t* w_out) {
    int nr = rounds_for_bits(bits);
    if (nr < 0) return ORACLE_ERR_KEYSIZE;
    if (!key || !w_out) return ORACLE_ERR_ARG;
    ensure_sbox();
    int nk = bits / 32;
    int total = 4 * (nr + 1);
    uint8_t (*w)[4] = (uint8_t (*)[4])w_out;
    for (int i = 0; i < nk; ++i)
        for (int j = 0; j < 4; ++j) w[i][j] = key[4 * i + j];
    uint8_t rcon = 0x01; /* Rcon[i/Nk] = x^(i/Nk - 1) */
    for (int i = nk; i < total; ++i) {
        uint8_t temp[4];
        memcpy(temp, w[i - 1], 4);
        if (i % nk == 0) {
            /* RotWord then SubWord, then XOR Rcon into the first byte */
            uint8_t t0 = temp[0];
            temp[0] = SBOX[temp[1]];
            temp[1] = SBOX[temp[2]];
            temp[2] = SBOX[temp[3]];
            temp[3] = SBOX[t0];
            temp[0] ^= rcon;
            rcon = xtime(rcon);
        } else if (nk > 6 && i % nk == 4) {
            for (int j = 0; j < 4; ++j) temp[j] = SBOX[temp[j]];
        }
        for (int j = 0; j < 4; ++j) w[i][j] = (uint8_t)(w[i - nk][j] ^ temp[j]);
    }
    return ORACLE_OK;
}

/* --------------------------------------------------------- round functions */

typedef uint8_t state_t[4][4];

static void add_round_key(state_t s, const uint8_t* rk /* 16 bytes */) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) s[r][c] ^= rk[4 * c + r];
}

static void sub_bytes(state_t s) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) s[r][c] = SBOX[s[r][c]];
}

static void inv_sub_bytes(state_t s) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) s[r][c] = INV_SBOX[s[r][c]];
}

/* Row r is rotated left by r positions (FIPS-197 5.1.2). */
static void shift_rows(state_t s) {
    for (int r = 1; r < 4; ++r) {
        uint8_t row[4];
        for (int c = 0; c < 4; ++c) row[c] = s[r][(c + r) % 4];
        for (int c = 0; c < 4; ++c) s[r][c] = row[c];
    }
}

/* Row r is rotated right by r positions (FIPS-197 5.3.1). */
static void inv_shift_rows(state_t s) {
    for (int r = 1; r < 4; ++r) {
        uint8_t row[4];
        for (int c = 0; c < 4; ++c) row[(c + r) % 4] = s[r][c];
        for (int c = 0; c < 4; ++c) s[r][c] = row[c];
    }
}

/* Each column is multiplied by {03}x^3+{01}x^2+{01}x+{02} (FIPS-197 5.1.3):
 * s'_r = 2*s_r ^ 3*s_{r+1} ^ s_{r+2} ^ s_{r+3}, with 3*a = xtime(a) ^ a. */
static void mix_columns(state_t s) {
    for (int c = 0; c < 4; ++c) {
        uint8_t a[4];
        for (int r = 0; r < 4; ++r) a[r] = s[r][c];
        for (int r = 0; r < 4; ++r) {
            uint8_t a0 = a[r], a1 = a[(r + 1) % 4], a2 = a[(r + 2) % 4], a3 = a[(r + 3) % 4];
            s[r][c] = (uint8_t)(xtime(a0) ^ (xtime(a1) ^ a1) ^ a2 ^ a3);
        }
    }
}

/* Inverse matrix rows {0e,0b,0d,09} circulant (FIPS-197 5.3.3). */
static void inv_mix_columns(state_t s) {
    for (int c = 0; c < 4; ++c) {
        uint8_t a[4];
        for (int r = 0; r < 4; ++r) a[r] = s[r][c];
        for (int r = 0; r < 4; ++r) {
            s[r][c] = (uint8_t)(oracle_gf_mul(a[r], 0x0e) ^ oracle_gf_mul(a[(r + 1) % 4], 0x0b) ^
                                oracle_gf_mul(a[(r + 2) % 4], 0x0d) ^ oracle_gf_mul(a[(r + 3) % 4], 0x09));
        }
    }
}

static void load_state(state_t s, const uint8_t* in) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) s[r][c] = in[r + 4 * c];
}

static void store_state(uint8_t* out, state_t s) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) out[r + 4 * c] = s[r][c];
}

/* Cipher (FIPS-197 5.1, Fig. 5). */
static void cipher_block(const uint8_t* in, uint8_t* out, const uint8_t* w, int nr) {
    state_t s;
    load_state(s, in);
    add_round_key(s, w);
    for (int round = 1; round < nr; ++round) {
        sub_bytes(s);
        shift_rows(s);
        mix_columns(s);
        add_round_key(s, w + 16 * round);
    }
    sub_bytes(s);
    shift_rows(s);
    add_round_key(s, w + 16 * nr);
    store_state(out, s);
}

/* InvCipher (FIPS-197 5.3, Fig. 12): the straight inverse order. */
static void inv_cipher_block(const uint8_t* in, uint8_t* out, const uint8_t* w, int nr) {
    state_t s;
    load_state(s, in);
    add_round_key(s, w + 16 * nr);
    for (int round = nr - 1; round >= 1; --round) {
        inv_shift_rows(s);
        inv_sub_bytes(s);
        add_round_key(s, w + 16 * round);
        inv_mix_columns(s);
    }
    inv_shift_rows(s);
    inv_sub_bytes(s);
    add_round_key(s, w);
    store_state(out, s);
}

/* ------------------------------------------------------------------ modes */

enum { MODE_ECB_ENC = 0, MODE_ECB_DEC = 1, MODE_CTR = 2, MODE_CBC_DEC = 3 };
enum { CTR_BE128 = 0, CTR_LE32_CARRY = 1 };

typedef struct {
    int mode;
    int nr;
    const uint8_t* w; /* expanded key, 16*(nr+1) bytes */
    const uint8_t* iv;
    int ctr_kind;
    const uint8_t* in;
    uint8_t* out;
    uint64_t first;    /* first block index of this worker's range */
    uint64_t count;    /* blocks in this worker's range */
} job_t;

/* Counter block for block index i.
 * CTR_BE128: the 16 IV bytes are one big-endian 128-bit integer; add i mod 2^128.
 * CTR_LE32_CARRY: the IV is four little-endian 32-bit words (x, y, z, w); add i
 *   to x and carry into y, z, w in turn (the paper's Section 3 counter, with the
 *   block index widened from 32 to 64 bits: its high half is added into y). */
static void counter_block(const uint8_t* iv, int kind, uint64_t i, uint8_t* ctr) {
    if (kind == CTR_BE128) {
        unsigned carry = 0;
        for (int b = 15; b >= 0; --b) {
            unsigned add = (15 - b) < 8 ? (unsigned)((i >> (8 * (15 - b))) & 0xff) : 0u;
            unsigned v = iv[b] + add + carry;
            ctr[b] = (uint8_t)v;
            carry = v >> 8;
        }
    } else {
        uint32_t word[4];
        for (int k = 0; k < 4; ++k)
            word[k] = (uint32_t)iv[4 * k] | ((uint32_t)iv[4 * k + 1] << 8) |
                      ((uint32_t)iv[4 * k + 2] << 16) | ((uint32_t)iv[4 * k + 3] << 24);
        uint64_t add[4] = {i & 0xffffffffu, i >> 32, 0, 0};
        uint64_t carry = 0;
        for (int k = 0; k < 4; ++k) {
            uint64_t v = (uint64_t)word[k] + add[k] + carry;
            word[k] = (uint32_t)v;
            carry = v >> 32;
        }
        for (int k = 0; k < 4; ++k)
            for (int b = 0; b < 4; ++b) ctr[4 * k + b] = (uint8_t)(word[k] >> (8 * b));
    }
}

static void run_job(const job_t* j) {
    for (uint64_t b = j->first; b < j->first + j->count; ++b) {
        const uint8_t* in = j->in + 16 * b;
        uint8_t* out = j->out + 16 * b;
        switch (j->mode) {
            case MODE_ECB_ENC:
                cipher_block(in, out, j->w, j->nr);
                break;
            case MODE_ECB_DEC:
                inv_cipher_block(in, out, j->w, j->nr);
                break;
            case MODE_CTR: {
                uint8_t ctr[16], ks[16];
                counter_block(j->iv, j->ctr_kind, b, ctr);
                cipher_block(ctr, ks, j->w, j->nr);
                for (int k = 0; k < 16; ++k) out[k] = (uint8_t)(in[k] ^ ks[k]);
                break;
            }
            case MODE_CBC_DEC: {
                uint8_t p[16];
                const uint8_t* prev = (b == 0) ? j->iv : (in - 16);
                inv_cipher_block(in, p, j->w, j->nr);
                for (int k = 0; k < 16; ++k) out[k] = (uint8_t)(p[k] ^ prev[k]);
                break;
            }
        }
    }
}

static void* worker(void* arg) {
    run_job((const job_t*)arg);
    return NULL;
}

/* Splits [0, nblocks) into nthreads contiguous ranges. CBC decryption reads
 * the input's previous block, so in == out is rejected for it (the read would
 * race with another worker's write). */
static int run_mode(int mode, const uint8_t* key, int bits, const uint8_t* iv, int ctr_kind,
                    const uint8_t* in, uint8_t* out, uint64_t nblocks, int nthreads) {
    int nr = rounds_for_bits(bits);
    if (nr < 0) return ORACLE_ERR_KEYSIZE;
    if (nblocks == 0) return ORACLE_OK;
    if (!key || !in || !out) return ORACLE_ERR_ARG;
    if ((mode == MODE_CTR || mode == MODE_CBC_DEC) && !iv) return ORACLE_ERR_ARG;
    if (mode == MODE_CBC_DEC && in == out) return ORACLE_ERR_ARG;
    uint8_t w[16 * 15];
    int rc = oracle_key_expansion(key, bits, w);
    if (rc) return rc;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > nblocks) nthreads = (int)nblocks;
    job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t* tids = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tids) {
        free(jobs);
        free(tids);
        return ORACLE_ERR_ARG;
    }
    uint64_t per = nblocks / (uint64_t)nthreads, extra = nblocks % (uint64_t)nthreads, at = 0;
    for (int t = 0; t < nthreads; ++t) {
        job_t j = {mode, nr, w, iv, ctr_kind, in, out, at, per + ((uint64_t)t < extra ? 1 : 0)};
        jobs[t] = j;
        at += jobs[t].count;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&tids[t], NULL, worker, &jobs[t]) != 0) break;
        started = t;
    }
    run_job(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tids[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) run_job(&jobs[t]); /* threads that failed to start */
    free(jobs);
    free(tids);
    return ORACLE_OK;
}

/* ECB encryption / decryption of nblocks independent 16-byte blocks (Section 3). */
int oracle_ecb(const uint8_t* key, int bits, int decrypt, const uint8_t* in, uint8_t* out,
               uint64_t nblocks, int nthreads) {
    return run_mode(decrypt ? MODE_ECB_DEC : MODE_ECB_ENC, key, bits, NULL, 0, in, out, nblocks,
                    nthreads);
}

/* CTR mode (Section 3): out_i = in_i XOR E_K(counter_i). */
int oracle_ctr(const uint8_t* key, int bits, const uint8_t* iv, int ctr_kind, const uint8_t* in,
               uint8_t* out, uint64_t nblocks, int nthreads) {
    if (ctr_kind != CTR_BE128 && ctr_kind != CTR_LE32_CARRY) return ORACLE_ERR_ARG;
    return run_mode(MODE_CTR, key, bits, iv, ctr_kind, in, out, nblocks, nthreads);
}

/* CBC decryption (Section 3, Eq. 2): out_i = D_K(in_i) XOR in_{i-1}, in_{-1} = IV. */
int oracle_cbc_decrypt(const uint8_t* key, int bits, const uint8_t* iv, const uint8_t* in,
                       uint8_t* out, uint64_t nblocks, int nthreads) {
    return run_mode(MODE_CBC_DEC, key, bits, iv, 0, in, out, nblocks, nthreads);
}

/* Counter block as the oracle forms it (exposed so tests can pin it). */
void oracle_counter_block(const uint8_t* iv, int ctr_kind, uint64_t i, uint8_t* ctr) {
    counter_block(iv, ctr_kind, i, ctr);
}
