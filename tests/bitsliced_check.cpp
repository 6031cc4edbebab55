// Test harness: runs the bitsliced cipher (csrc/bitsliced.h) on the CPU for
// 32 blocks so its logic can be compared with the oracle without a GPU.  The
// state is split between two halves as in the kernel, each half run by its own
// host thread; the lane shuffle of the kernel becomes a read of the other
// thread's copy of the plane between two barriers.
// stdin: bits (int32), decrypt (int32), 4*(Nr+1) encryption round-key words,
// 32 blocks of 16 bytes.  stdout: the 32 output blocks.
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>

#include "bitsliced.h"

namespace {

struct Barrier2 {
    std::mutex mu;
    std::condition_variable cv;
    int waiting = 0;
    unsigned gen = 0;
    void wait() {
        std::unique_lock<std::mutex> lk(mu);
        const unsigned g = gen;
        if (++waiting == 2) {
            waiting = 0;
            ++gen;
            cv.notify_all();
        } else {
            cv.wait(lk, [&] { return gen != g; });
        }
    }
};

struct Exchange {
    Barrier2 bar;
    uint32_t slot[2][64];
};

// The other half's plane p: both halves post theirs, then read the other's.
struct ThreadPair {
    Exchange* x;
    int h;
    uint32_t operator()(uint32_t v, int p) const {
        x->slot[h][p] = v;
        x->bar.wait();
        const uint32_t r = x->slot[1 - h][p];
        x->bar.wait();
        return r;
    }
};

template <int NR>
void run_half(uint32_t (&s)[64], const gbaes::bs::HalfKeys& keys, bool dec, Exchange* x, int h) {
    if (dec)
        gbaes::bs::decrypt_half<NR>(s, keys, ThreadPair{x, h});
    else
        gbaes::bs::encrypt_half<NR>(s, keys, ThreadPair{x, h});
}

}  // namespace

int main() {
    int32_t hdr[2];
    if (fread(hdr, 4, 2, stdin) != 2) return 1;
    const int bits = hdr[0], dec = hdr[1];
    const int nr = bits == 128 ? 10 : bits == 192 ? 12 : 14;
    uint32_t rk[60];
    if (fread(rk, 4, 4 * (nr + 1), stdin) != (size_t)(4 * (nr + 1))) return 1;
    uint32_t blocks[32][4];
    if (fread(blocks, 16, 32, stdin) != 32) return 1;
    static uint32_t planes[15][128];
    static uint32_t split[15 * gbaes::bs::kKeyStepWords];
    gbaes::bs::make_key_planes(rk, nr, dec != 0, planes);
    gbaes::bs::split_key_planes(planes, nr, split);
    static uint32_t s[2][64];
    for (int h = 0; h < 2; ++h) {  // half h: words 2h, 2h+1 of every block, as the kernel loads them
        for (int k = 0; k < 32; ++k) {
            s[h][k] = blocks[k][2 * h];
            s[h][32 + k] = blocks[k][2 * h + 1];
        }
        gbaes::bs::transpose32(&s[h][0]);
        gbaes::bs::transpose32(&s[h][32]);
    }
    static Exchange x;
    auto work = [&](int h) {
        const gbaes::bs::HalfKeys keys{split + gbaes::bs::kKeyHalfWords * h};
        switch (nr) {
            case 10: run_half<10>(s[h], keys, dec != 0, &x, h); break;
            case 12: run_half<12>(s[h], keys, dec != 0, &x, h); break;
            default: run_half<14>(s[h], keys, dec != 0, &x, h); break;
        }
    };
    std::thread t1(work, 1);
    work(0);
    t1.join();
    for (int h = 0; h < 2; ++h) {
        gbaes::bs::transpose32(&s[h][0]);
        gbaes::bs::transpose32(&s[h][32]);
        for (int k = 0; k < 32; ++k) {
            blocks[k][2 * h] = s[h][k];
            blocks[k][2 * h + 1] = s[h][32 + k];
        }
    }
    fwrite(blocks, 16, 32, stdout);
    return 0;
}
