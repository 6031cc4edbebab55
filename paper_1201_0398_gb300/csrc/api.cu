// The C ABI (include/gbaes.h): key contexts, argument checks and dispatch.
#include <cuda.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "aes_tables.h"
#include "gbaes_internal.h"

namespace gbaes {

// ------------------------------------------------------------------ errors

static thread_local char t_error[512];

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_error, sizeof t_error, fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { t_error[0] = '\0'; }

// ------------------------------------------------------------ key schedule

static int rounds_for(int bits) { return bits == 128 ? 10 : bits == 192 ? 12 : bits == 256 ? 14 : -1; }

static uint32_t sub_word(uint32_t w) {
    const uint8_t* s = kAesTables.sbox;
    return (uint32_t)s[w & 0xff] | ((uint32_t)s[(w >> 8) & 0xff] << 8) | ((uint32_t)s[(w >> 16) & 0xff] << 16) |
           ((uint32_t)s[w >> 24] << 24);
}

// InvMixColumns of one column held as a little-endian word (row r = byte r).
static uint32_t inv_mix_word(uint32_t w) {
    uint8_t a[4] = {(uint8_t)w, (uint8_t)(w >> 8), (uint8_t)(w >> 16), (uint8_t)(w >> 24)};
    static const uint8_t row0[4] = {0x0e, 0x0b, 0x0d, 0x09};
    uint32_t out = 0;
    for (int r = 0; r < 4; ++r) {
        uint8_t v = 0;
        for (int k = 0; k < 4; ++k) v ^= gf_mul_log(a[k], row0[(k - r + 4) & 3]);
        out |= (uint32_t)v << (8 * r);
    }
    return out;
}

// Word-oriented KeyExpansion on little-endian words: RotWord is a right
// rotation by 8 bits, Rcon is XORed into the low byte.
static int expand(const uint8_t* key, int bits, uint32_t* enc, uint32_t* dec) {
    const int nr = rounds_for(bits);
    if (nr < 0) return fail(AES_ERR_KEYSIZE, "key size %d bits is not 128, 192 or 256", bits);
    if (!key) return fail(AES_ERR_ARG, "key is NULL");
    const int nk = bits / 32, total = 4 * (nr + 1);
    uint32_t w[60];
    for (int i = 0; i < nk; ++i)
        w[i] = (uint32_t)key[4 * i] | ((uint32_t)key[4 * i + 1] << 8) | ((uint32_t)key[4 * i + 2] << 16) |
               ((uint32_t)key[4 * i + 3] << 24);
    uint8_t rcon = 1;
    for (int i = nk; i < total; ++i) {
        uint32_t t = w[i - 1];
        if (i % nk == 0) {
            t = sub_word((t >> 8) | (t << 24)) ^ rcon;
            rcon = gf_mul_log(rcon, 2);
        } else if (nk == 8 && i % nk == 4) {
            t = sub_word(t);
        }
        w[i] = w[i - nk] ^ t;
    }
    if (enc) memcpy(enc, w, sizeof(uint32_t) * total);
    if (dec) {
        // Equivalent inverse cipher: round r uses enc round Nr-r, with
        // InvMixColumns applied for 1 <= r <= Nr-1.
        for (int r = 0; r <= nr; ++r)
            for (int j = 0; j < 4; ++j) {
                uint32_t k = w[4 * (nr - r) + j];
                dec[4 * r + j] = (r == 0 || r == nr) ? k : inv_mix_word(k);
            }
    }
    return nr;
}

// ------------------------------------------------------------- device info

static std::mutex g_dev_mu;
static DeviceInfo g_dev[64];
static bool g_dev_ok[64];
typedef CUresult (*PointerAttrsFn)(unsigned int, CUpointer_attribute*, void**, CUdeviceptr);
static PointerAttrsFn g_ptr_attrs = nullptr;
static bool g_ptr_attrs_tried = false;

int current_device_info(DeviceInfo* info) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(AES_ERR_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_dev_ok[dev]) {
        DeviceInfo d{};
        d.device = dev;
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.pageable_access, cudaDevAttrPageableMemoryAccess, dev);
        if (e != cudaSuccess) return fail(AES_ERR_CUDA, "device attributes: %s", cudaGetErrorString(e));
        g_dev[dev] = d;
        g_dev_ok[dev] = true;
    }
    *info = g_dev[dev];
    return AES_OK;
}

// The CUDA context current on this thread, as an id that is unique for the
// process's life (a handle value can be reused once a context is destroyed, an
// id cannot).  Per-context state -- a kernel's shared-memory attribute, the
// device address of a __device__ symbol -- belongs to the module loaded in one
// context, so it is cached by this id, not by device index: a caller may make
// its own context current, and cudaDeviceReset replaces the primary context.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
static CtxGetCurrentFn g_ctx_current = nullptr;
static CtxGetIdFn g_ctx_get_id = nullptr;
static bool g_ctx_fns_tried = false;

static void* driver_fn(const char* name) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return fn;
    return nullptr;
}

int current_context_id(unsigned long long* id) {
    {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        if (!g_ctx_fns_tried) {
            g_ctx_fns_tried = true;
            g_ctx_current = (CtxGetCurrentFn)driver_fn("cuCtxGetCurrent");
            g_ctx_get_id = (CtxGetIdFn)driver_fn("cuCtxGetId");
        }
    }
    if (!g_ctx_current || !g_ctx_get_id) return fail(AES_ERR_CUDA, "cuCtxGetCurrent/cuCtxGetId unavailable");
    CUcontext c = nullptr;
    if (g_ctx_current(&c) != CUDA_SUCCESS) return fail(AES_ERR_CUDA, "cuCtxGetCurrent failed");
    if (!c) {
        // Nothing current yet: cudaSetDevice makes the device's primary context
        // current (it allocates nothing).
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess) return fail(AES_ERR_CUDA, "no CUDA context: %s", cudaGetErrorString(e));
        if (g_ctx_current(&c) != CUDA_SUCCESS || !c) return fail(AES_ERR_CUDA, "no current CUDA context");
    }
    if (g_ctx_get_id(c, id) != CUDA_SUCCESS) return fail(AES_ERR_CUDA, "cuCtxGetId failed");
    return AES_OK;
}

int set_max_dynamic_smem(const void* fn, int bytes) {
    unsigned long long ctx = 0;
    int rc = current_context_id(&ctx);
    if (rc) return rc;
    static std::mutex mu;
    static std::set<std::pair<const void*, unsigned long long>> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({fn, ctx})) return AES_OK;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return fail(AES_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    done.insert({fn, ctx});
    return AES_OK;
}

static PointerAttrsFn pointer_attrs_fn() {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_ptr_attrs_tried) {
        g_ptr_attrs_tried = true;
        g_ptr_attrs = (PointerAttrsFn)driver_fn("cuPointerGetAttributes");
    }
    return g_ptr_attrs;
}

// Accepts device, managed and page-locked host memory whose allocation holds
// all of [p, p+bytes); fails closed when the allocation's extent cannot be read.
// Unregistered pageable host memory is refused even where the GPU could read
// it, because its extent cannot be checked before the launch.  One driver call
// reads the memory type, the managed flag, the device address and the extent.
static int check_device_range_ex(const void* p, size_t bytes, const char* what, uintptr_t* alloc_lo,
                                 uintptr_t* alloc_hi) {
    if (!p) return fail(AES_ERR_ARG, "%s is NULL", what);
    if (((uintptr_t)p & 15u) != 0) return fail(AES_ERR_ALIGN, "%s (%p) is not 16-byte aligned", what, p);
    PointerAttrsFn get = pointer_attrs_fn();
    if (!get) return fail(AES_ERR_CUDA, "cuPointerGetAttributes unavailable: cannot check the extent of %s", what);
    unsigned int mem_type = 0, is_managed = 0;
    CUdeviceptr dev_ptr = 0, start = 0;
    size_t size = 0;
    CUpointer_attribute attrs[5] = {CU_POINTER_ATTRIBUTE_MEMORY_TYPE, CU_POINTER_ATTRIBUTE_IS_MANAGED,
                                    CU_POINTER_ATTRIBUTE_DEVICE_POINTER, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR,
                                    CU_POINTER_ATTRIBUTE_RANGE_SIZE};
    void* data[5] = {&mem_type, &is_managed, &dev_ptr, &start, &size};
    if (get(5, attrs, data, (CUdeviceptr)p) != CUDA_SUCCESS)
        return fail(AES_ERR_ARG, "%s (%p): not a pointer CUDA knows", what, p);
    const bool device = mem_type == CU_MEMORYTYPE_DEVICE || mem_type == CU_MEMORYTYPE_UNIFIED || is_managed;
    const bool pinned = mem_type == CU_MEMORYTYPE_HOST;
    if (!device && !pinned)
        return fail(AES_ERR_ARG, "%s (%p) is not device, managed or page-locked host memory", what, p);
    if (pinned && dev_ptr != (CUdeviceptr)p)
        return fail(AES_ERR_ARG, "%s (%p): page-locked memory is not mapped at the same device address", what, p);
    if (size == 0) return fail(AES_ERR_ARG, "%s (%p): the extent of its allocation cannot be read", what, p);
    const uintptr_t lo = (uintptr_t)p, end = (uintptr_t)start + size;
    if (lo < (uintptr_t)start || lo > end || bytes > end - lo)
        return fail(AES_ERR_ARG, "%s: %zu bytes at %p run past the end of its allocation (%zu bytes left)", what,
                    bytes, p, lo <= end ? (size_t)(end - lo) : (size_t)0);
    *alloc_lo = (uintptr_t)start;
    *alloc_hi = end;
    return AES_OK;
}

int check_device_range(const void* p, size_t bytes, const char* what) {
    uintptr_t lo = 0, hi = 0;
    return check_device_range_ex(p, bytes, what, &lo, &hi);
}

int check_device_range_cached(const void* p, size_t bytes, const char* what, RangeCache* cache) {
    if (!cache) return check_device_range(p, bytes, what);
    const uintptr_t a = (uintptr_t)p;
    if (p && (a & 15u) == 0)
        for (int i = 0; i < cache->n; ++i)
            if (a >= cache->lo[i] && a <= cache->hi[i] && bytes <= cache->hi[i] - a) return AES_OK;
    uintptr_t lo = 0, hi = 0;
    const int rc = check_device_range_ex(p, bytes, what, &lo, &hi);
    if (rc == AES_OK) {  // remember the allocation (the oldest entry makes room)
        const int k = cache->n < RangeCache::kSize ? cache->n++ : (cache->next++ % RangeCache::kSize);
        cache->lo[k] = lo;
        cache->hi[k] = hi;
    }
    return rc;
}

// ------------------------------------------------------- launch defaults

struct Tuning {
    int threads;
    int bpt;
};
static std::atomic<int> g_kernel{AES_KERNEL_TABLE};
static Tuning g_tuning[3][2] = {{{1024, 2}, {1024, 2}}, {{1024, 2}, {1024, 2}}, {{1024, 2}, {1024, 2}}};
static std::mutex g_tuning_mu;

static int bits_index(int bits) { return bits == 128 ? 0 : bits == 192 ? 1 : bits == 256 ? 2 : -1; }

static Tuning get_tuning(int bits, int decrypt) {
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    return g_tuning[bits_index(bits)][decrypt ? 1 : 0];
}

int table_default_shape(int bits, int decrypt, int* threads, int* bpt) {
    if (bits_index(bits) < 0) return fail(AES_ERR_KEYSIZE, "key size %d bits is not 128, 192 or 256", bits);
    Tuning t = get_tuning(bits, decrypt);
    *threads = t.threads;
    *bpt = t.bpt;
    return AES_OK;
}

static bool valid_threads(int t) { return t >= 64 && t <= 1024 && t % 32 == 0; }
static bool valid_bpt(int b) { return b == 1 || b == 2 || b == 4; }
static bool valid_kernel(int k) {
    return k == AES_KERNEL_TABLE || k == AES_KERNEL_BITSLICED || k == AES_KERNEL_TABLE_COMPACT ||
           k == AES_KERNEL_TABLE_REPLICATED;
}

static int check_ctx(const aes_ctx* ctx) {
    if (!ctx || ctx->magic != kCtxMagic) return fail(AES_ERR_ARG, "invalid or freed aes_ctx");
    return AES_OK;
}

// Range checks common to the block calls.  allow_inplace: in == out permitted.
static int check_io(const void* in, const void* out, size_t nblocks, bool allow_inplace) {
    if (nblocks > (SIZE_MAX >> 4)) return fail(AES_ERR_ARG, "nblocks %zu overflows the byte count", nblocks);
    const size_t bytes = nblocks * 16;
    // Cheap checks on both pointers before any driver query.
    if (!in) return fail(AES_ERR_ARG, "in is NULL");
    if (!out) return fail(AES_ERR_ARG, "out is NULL");
    if (((uintptr_t)in | (uintptr_t)out) & 15u) return fail(AES_ERR_ALIGN, "in and out must be 16-byte aligned");
    int rc = check_device_range(in, bytes, "in");
    if (rc) return rc;
    rc = check_device_range(out, bytes, "out");
    if (rc) return rc;
    const uintptr_t i0 = (uintptr_t)in, o0 = (uintptr_t)out;
    if (i0 == o0) {
        if (!allow_inplace) return fail(AES_ERR_ARG, "in and out must not overlap for this mode");
        return AES_OK;
    }
    if (i0 < o0 + bytes && o0 < i0 + bytes) return fail(AES_ERR_ARG, "in and out overlap partially");
    return AES_OK;
}

static int run_block_op(const aes_ctx* ctx, Mode mode, const void* in, void* out, size_t nblocks, int kernel,
                        int threads, int bpt, void* stream, const uint8_t* iv, int ctr_kind, uint64_t first) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (nblocks == 0) return AES_OK;
    rc = check_io(in, out, nblocks, mode != kCbcDec);
    if (rc) return rc;
    EcbArgs a;
    memset(&a, 0, sizeof a);
    a.in = (const uint4*)in;
    a.out = (uint4*)out;
    a.nblocks = nblocks;
    const bool dec = (mode == kDec || mode == kCbcDec);
    memcpy(a.rk, dec ? ctx->dec_rk : ctx->enc_rk, sizeof(uint32_t) * 4 * (ctx->nr + 1));
    if (mode == kCtr) {
        uint64_t hi = 0, lo = 0;
        if (ctr_kind == AES_CTR_BE128) {
            for (int b = 0; b < 8; ++b) hi = (hi << 8) | iv[b];
            for (int b = 8; b < 16; ++b) lo = (lo << 8) | iv[b];
        } else {
            for (int b = 7; b >= 0; --b) lo = (lo << 8) | iv[b];
            for (int b = 15; b >= 8; --b) hi = (hi << 8) | iv[b];
        }
        a.ctr_lo = lo;
        a.ctr_hi = hi;
        a.ctr_be = ctr_kind == AES_CTR_BE128;
        a.first = first;
    }
    if (mode == kCbcDec) memcpy(a.iv, iv, 16);
    if (kernel == AES_KERNEL_BITSLICED) {
        if (mode != kEnc && mode != kDec) return fail(AES_ERR_ARG, "the bitsliced kernel implements ECB only");
        return launch_bitsliced(a, ctx->enc_rk, ctx->nr, mode, threads, (cudaStream_t)stream);
    }
    return launch_table(a, ctx->nr, mode, threads, bpt, kernel, (cudaStream_t)stream);
}

}  // namespace gbaes

using namespace gbaes;

extern "C" {

aes_ctx* aes_expand_key(const uint8_t* key, int bits) {
    aes_ctx* c = (aes_ctx*)calloc(1, sizeof(aes_ctx));
    if (!c) {
        fail(AES_ERR_NOMEM, "out of host memory");
        return nullptr;
    }
    int nr = expand(key, bits, c->enc_rk, c->dec_rk);
    if (nr < 0) {
        free(c);
        return nullptr;
    }
    c->magic = kCtxMagic;
    c->bits = bits;
    c->nr = nr;
    return c;
}

void aes_free_ctx(aes_ctx* ctx) {
    if (!ctx) return;
    ctx->magic = 0;
    free(ctx);
}

int aes_ctx_bits(const aes_ctx* ctx) {
    int rc = check_ctx(ctx);
    return rc ? rc : ctx->bits;
}

int aes_encrypt_ecb(const aes_ctx* ctx, const void* in, void* out, size_t nblocks, void* stream) {
    if (check_ctx(ctx)) return AES_ERR_ARG;
    Tuning t = get_tuning(ctx->bits, 0);
    return run_block_op(ctx, kEnc, in, out, nblocks, g_kernel.load(), t.threads, t.bpt, stream, nullptr, 0, 0);
}

int aes_decrypt_ecb(const aes_ctx* ctx, const void* in, void* out, size_t nblocks, void* stream) {
    if (check_ctx(ctx)) return AES_ERR_ARG;
    Tuning t = get_tuning(ctx->bits, 1);
    return run_block_op(ctx, kDec, in, out, nblocks, g_kernel.load(), t.threads, t.bpt, stream, nullptr, 0, 0);
}

int aes_ecb_ex(const aes_ctx* ctx, int decrypt, const void* in, void* out, size_t nblocks, int kernel, int threads,
               int blocks_per_thread, void* stream) {
    if (check_ctx(ctx)) return AES_ERR_ARG;
    if (decrypt != 0 && decrypt != 1) return fail(AES_ERR_ARG, "decrypt must be 0 or 1");
    if (!valid_kernel(kernel)) return fail(AES_ERR_ARG, "unknown kernel %d", kernel);
    Tuning t = get_tuning(ctx->bits, decrypt);
    if (threads == 0) threads = kernel == AES_KERNEL_BITSLICED ? 256 : t.threads;
    if (blocks_per_thread == 0) blocks_per_thread = t.bpt;
    if (!valid_threads(threads)) return fail(AES_ERR_ARG, "threads %d: need a multiple of 32 in [64, 1024]", threads);
    if (kernel != AES_KERNEL_BITSLICED && !valid_bpt(blocks_per_thread))
        return fail(AES_ERR_ARG, "blocks_per_thread %d: need 1, 2 or 4", blocks_per_thread);
    return run_block_op(ctx, decrypt ? kDec : kEnc, in, out, nblocks, kernel, threads, blocks_per_thread, stream,
                        nullptr, 0, 0);
}

int aes_ctr_xcrypt(const aes_ctx* ctx, const uint8_t* iv, int counter_kind, uint64_t first_block, const void* in,
                   void* out, size_t nblocks, void* stream) {
    if (check_ctx(ctx)) return AES_ERR_ARG;
    if (!iv) return fail(AES_ERR_ARG, "iv is NULL");
    if (counter_kind != AES_CTR_BE128 && counter_kind != AES_CTR_LE32_CARRY)
        return fail(AES_ERR_ARG, "unknown counter kind %d", counter_kind);
    if (nblocks > 0 && first_block > UINT64_MAX - (uint64_t)(nblocks - 1))
        return fail(AES_ERR_ARG, "first_block + nblocks exceeds 2^64 block indices");
    Tuning t = get_tuning(ctx->bits, 0);
    return run_block_op(ctx, kCtr, in, out, nblocks, AES_KERNEL_TABLE, t.threads, t.bpt, stream, iv, counter_kind,
                        first_block);
}

int aes_cbc_decrypt(const aes_ctx* ctx, const uint8_t* iv, const void* in, void* out, size_t nblocks, void* stream) {
    if (check_ctx(ctx)) return AES_ERR_ARG;
    if (!iv) return fail(AES_ERR_ARG, "iv is NULL");
    Tuning t = get_tuning(ctx->bits, 1);
    return run_block_op(ctx, kCbcDec, in, out, nblocks, AES_KERNEL_TABLE, t.threads, t.bpt, stream, iv, 0, 0);
}

int aes_set_kernel(int which) {
    if (!valid_kernel(which)) return fail(AES_ERR_ARG, "unknown kernel %d", which);
    return g_kernel.exchange(which);
}

int aes_set_tuning(int bits, int decrypt, int threads, int blocks_per_thread) {
    int bi = bits_index(bits);
    if (bi < 0) return fail(AES_ERR_KEYSIZE, "key size %d bits is not 128, 192 or 256", bits);
    if (decrypt != 0 && decrypt != 1) return fail(AES_ERR_ARG, "decrypt must be 0 or 1");
    if (!valid_threads(threads)) return fail(AES_ERR_ARG, "threads %d: need a multiple of 32 in [64, 1024]", threads);
    if (!valid_bpt(blocks_per_thread)) return fail(AES_ERR_ARG, "blocks_per_thread %d: need 1, 2 or 4", blocks_per_thread);
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    g_tuning[bi][decrypt] = Tuning{threads, blocks_per_thread};
    return AES_OK;
}

int aes_device_status(int clear) { return read_device_status(clear); }

const char* aes_last_error(void) { return t_error; }

int aes_key_schedule(const uint8_t* key, int bits, uint32_t* enc_rk, uint32_t* dec_rk) {
    return expand(key, bits, enc_rk, dec_rk);
}

int aes_host_tables(uint32_t* te0, uint32_t* td0, uint8_t* sbox, uint8_t* inv_sbox) {
    if (te0) memcpy(te0, kAesTables.te0, sizeof kAesTables.te0);
    if (td0) memcpy(td0, kAesTables.td0, sizeof kAesTables.td0);
    if (sbox) memcpy(sbox, kAesTables.sbox, 256);
    if (inv_sbox) memcpy(inv_sbox, kAesTables.inv_sbox, 256);
    return AES_OK;
}

}  // extern "C"
