/* Plain C user of the C ABI (include/gbaes.h): no Python, no torch.
 * Encrypts and decrypts 1 MiB with each key size through device buffers from
 * cudaMalloc, checks the round trip and the error codes of bad arguments,
 * prints the first ciphertext block of each key size for the test to compare
 * with the oracle, and runs requests through the resident server and back.
 * Exit status 0 on success. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "gbaes.h"

#define CHECK(cond, msg)                                                      \
    do {                                                                      \
        if (!(cond)) {                                                        \
            fprintf(stderr, "FAIL: %s (%s)\n", msg, aes_last_error());        \
            return 1;                                                         \
        }                                                                     \
    } while (0)

int main(void) {
    const size_t nblocks = 65536, bytes = nblocks * 16;
    unsigned char* host = (unsigned char*)malloc(bytes);
    unsigned char* back = (unsigned char*)malloc(bytes);
    for (size_t i = 0; i < bytes; ++i) host[i] = (unsigned char)(i * 131u + 7u);
    void *d_in = NULL, *d_out = NULL;
    CHECK(cudaMalloc(&d_in, bytes) == cudaSuccess && cudaMalloc(&d_out, bytes) == cudaSuccess, "cudaMalloc");
    cudaStream_t s;
    CHECK(cudaStreamCreate(&s) == cudaSuccess, "stream");
    const int sizes[3] = {128, 192, 256};
    for (int t = 0; t < 3; ++t) {
        unsigned char key[32];
        for (int i = 0; i < 32; ++i) key[i] = (unsigned char)(i + 16 * t);
        aes_ctx* k = aes_expand_key(key, sizes[t]);
        CHECK(k != NULL && aes_ctx_bits(k) == sizes[t], "aes_expand_key");
        CHECK(cudaMemcpy(d_in, host, bytes, cudaMemcpyHostToDevice) == cudaSuccess, "copy in");
        CHECK(aes_encrypt_ecb(k, d_in, d_out, nblocks, s) == AES_OK, "aes_encrypt_ecb");
        CHECK(aes_decrypt_ecb(k, d_out, d_in, nblocks, s) == AES_OK, "aes_decrypt_ecb");
        CHECK(cudaStreamSynchronize(s) == cudaSuccess, "sync");
        CHECK(cudaMemcpy(back, d_in, bytes, cudaMemcpyDeviceToHost) == cudaSuccess, "copy back");
        CHECK(memcmp(back, host, bytes) == 0, "decrypt(encrypt(x)) != x");
        unsigned char first[16];
        CHECK(cudaMemcpy(first, d_out, 16, cudaMemcpyDeviceToHost) == cudaSuccess, "copy first block");
        printf("%d ", sizes[t]);
        for (int i = 0; i < 16; ++i) printf("%02x", first[i]);
        printf("\n");
        /* bad arguments are error codes, not faults */
        CHECK(aes_encrypt_ecb(k, (char*)d_in + 1, d_out, 4, s) == AES_ERR_ALIGN, "misaligned in");
        CHECK(aes_encrypt_ecb(k, d_in, d_out, nblocks + 1, s) == AES_ERR_ARG, "range past the allocation");
        CHECK(aes_encrypt_ecb(k, host, d_out, 4, s) == AES_ERR_ARG, "pageable host pointer");
        CHECK(aes_encrypt_ecb(k, d_in, d_out, 0, s) == AES_OK, "empty input");
        aes_free_ctx(k);
    }
    CHECK(aes_expand_key((const unsigned char*)"0123456789abcdef", 100) == NULL, "bad key size");

    /* The resident server from C: 64 requests of 1,024 blocks, alternating
     * directions, on disjoint slices; every request completes, and decrypting
     * the encrypted slices with a second pass gives the input back. */
    {
        unsigned char key[16];
        for (int i = 0; i < 16; ++i) key[i] = (unsigned char)(3 * i + 1);
        aes_ctx* k = aes_expand_key(key, 128);
        CHECK(k != NULL, "server key");
        CHECK(cudaMemcpy(d_in, host, bytes, cudaMemcpyHostToDevice) == cudaSuccess, "copy in");
        CHECK(cudaDeviceSynchronize() == cudaSuccess, "sync before the server");
        aes_server_config cfg;
        memset(&cfg, 0, sizeof cfg);
        cfg.flags = AES_SERVER_RESIDENT;
        const aes_ctx* keys[1] = {k};
        for (int pass = 0; pass < 2; ++pass) {
            aes_server* srv = aes_server_create(keys, 1, &cfg);
            CHECK(srv != NULL, "aes_server_create");
            for (int i = 0; i < 64; ++i) {
                aes_server_request r;
                memset(&r, 0, sizeof r);
                r.id = (uint64_t)i;
                r.nblocks = 1024;
                r.key_index = 0;
                r.decrypt = (uint32_t)((i + pass) & 1); /* the second pass undoes the first */
                r.in = (const char*)(pass ? d_out : d_in) + (size_t)i * 1024 * 16;
                r.out = (char*)(pass ? d_in : d_out) + (size_t)i * 1024 * 16;
                CHECK(aes_server_submit(srv, &r) == AES_OK, "aes_server_submit");
            }
            CHECK(aes_server_drain(srv, 10.0) == AES_OK, "aes_server_drain");
            aes_server_completion c[64];
            int got = 0, ok = 0;
            for (int n; (n = aes_server_poll(srv, c, 64)) > 0;) {
                for (int i = 0; i < n; ++i) ok += c[i].status == AES_OK;
                got += n;
            }
            CHECK(got == 64 && ok == 64, "every request completes");
            aes_server_stats st;
            CHECK(aes_server_get_stats(srv, &st) == AES_OK && st.completed == 64, "server stats");
            aes_server_destroy(srv);
        }
        CHECK(cudaMemcpy(back, d_in, bytes, cudaMemcpyDeviceToHost) == cudaSuccess, "copy back");
        CHECK(memcmp(back, host, 64 * 1024 * 16) == 0, "server: second pass did not undo the first");
        aes_free_ctx(k);
    }
    CHECK(aes_device_status(0) == 0, "device status");
    cudaFree(d_in);
    cudaFree(d_out);
    cudaStreamDestroy(s);
    free(host);
    free(back);
    printf("c abi ok\n");
    return 0;
}
