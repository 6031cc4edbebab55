// Test harness: runs the bitsliced circuit (csrc/bitsliced.h) on the CPU for
// 32 blocks so its logic can be compared with the oracle without a GPU.
// stdin: bits (int32), decrypt (int32), 4*(Nr+1) encryption round-key words,
// 32 blocks of 16 bytes.  stdout: the 32 output blocks.
#include <cstdio>
#include <cstring>

#include "bitsliced.h"

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
    gbaes::bs::make_key_planes(rk, nr, dec != 0, planes);
    const gbaes::bs::PlaneKeys keys{planes};
    uint32_t s[128];
    for (int k = 0; k < 32; ++k)
        for (int i = 0; i < 4; ++i) s[32 * i + k] = blocks[k][i];
    for (int i = 0; i < 4; ++i) gbaes::bs::transpose32(&s[32 * i]);
    switch (nr * 2 + dec) {
        case 20: gbaes::bs::encrypt_planes<10>(s, keys); break;
        case 21: gbaes::bs::decrypt_planes<10>(s, keys); break;
        case 24: gbaes::bs::encrypt_planes<12>(s, keys); break;
        case 25: gbaes::bs::decrypt_planes<12>(s, keys); break;
        case 28: gbaes::bs::encrypt_planes<14>(s, keys); break;
        default: gbaes::bs::decrypt_planes<14>(s, keys); break;
    }
    for (int i = 0; i < 4; ++i) gbaes::bs::transpose32(&s[32 * i]);
    for (int k = 0; k < 32; ++k)
        for (int i = 0; i < 4; ++i) blocks[k][i] = s[32 * i + k];
    fwrite(blocks, 16, 32, stdout);
    return 0;
}
