/*
 * aes_client.c -- a plain C99 user of the library's C ABI (include/aesgb.h),
 * compiled and run by tests/test_c_client.py.
 *
 *   aes_client keys <hexkey>
 *       expand the key (FIPS-197 5.2) and print Nr, then rk_enc and rk_dec as
 *       hex byte strings, one line each; no device is used.
 *   aes_client errors
 *       print the status of a few invalid calls, one per line.
 *   aes_client ecb <hexkey> <infile> <encfile> <decfile>
 *       encrypt the whole blocks of infile on the device (aes_ecb_encrypt),
 *       write the ciphertext, decrypt it in place (aes_ecb_decrypt) and write
 *       the result.
 * Exit status 0 on success; a failed call prints its status and exits 1.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "aesgb.h"

static int parse_key(const char *hex, uint8_t *key) {
    size_t n = strlen(hex), i;
    if (n != 32 && n != 48 && n != 64) return -1;
    for (i = 0; i < n / 2; ++i) {
        unsigned int b;
        if (sscanf(hex + 2 * i, "%2x", &b) != 1) return -1;
        key[i] = (uint8_t)b;
    }
    return (int)(n * 4);
}

static void print_words(const uint32_t *w, int nwords) {
    const uint8_t *b = (const uint8_t *)w;
    int i;
    for (i = 0; i < 4 * nwords; ++i) printf("%02x", b[i]);
    printf("\n");
}

static int check(int st, const char *what) {
    if (st < 0) {
        fprintf(stderr, "%s: %s\n", what, aes_status_str(st));
        exit(1);
    }
    return st;
}

static int cmd_keys(const char *hex) {
    uint8_t key[32];
    uint32_t enc[60], dec[60];
    int nr;
    const int bits = parse_key(hex, key);
    if (bits < 0) return 2;
    nr = check(aes_expand_key(bits, key, enc, dec), "aes_expand_key");
    printf("%d\n", nr);
    print_words(enc, 4 * (nr + 1));
    print_words(dec, 4 * (nr + 1));
    return 0;
}

static int cmd_errors(void) {
    uint8_t key[16] = {0};
    uint32_t enc[60];
    printf("%d\n", aes_expand_key(100, key, enc, NULL));
    printf("%d\n", aes_expand_key(128, NULL, enc, NULL));
    /* nrounds is checked before the (never dereferenced) buffer addresses */
    printf("%d\n", aes_ecb_encrypt(enc, 11, (const uint8_t *)(uintptr_t)0x100000, (uint8_t *)(uintptr_t)0x200000,
                                    1, NULL));
    printf("%s\n", aes_status_str(AES_E_OVERLAP));
    return 0;
}

static uint8_t *read_file(const char *path, size_t *len) {
    FILE *f = fopen(path, "rb");
    uint8_t *buf;
    long n;
    if (!f) return NULL;
    fseek(f, 0, SEEK_END);
    n = ftell(f);
    fseek(f, 0, SEEK_SET);
    buf = (uint8_t *)malloc(n > 0 ? (size_t)n : 1);
    if (buf && n > 0 && fread(buf, 1, (size_t)n, f) != (size_t)n) {
        free(buf);
        buf = NULL;
    }
    fclose(f);
    *len = n > 0 ? (size_t)n : 0;
    return buf;
}

static int write_file(const char *path, const uint8_t *buf, size_t len) {
    FILE *f = fopen(path, "wb");
    int ok;
    if (!f) return -1;
    ok = fwrite(buf, 1, len, f) == len;
    return fclose(f) == 0 && ok ? 0 : -1;
}

static int cmd_ecb(const char *hex, const char *in_path, const char *enc_path, const char *dec_path) {
    uint8_t key[32], *host, *dev = NULL;
    uint32_t enc[60], dec[60];
    size_t len, nblocks;
    int nr;
    const int bits = parse_key(hex, key);
    if (bits < 0) return 2;
    nr = check(aes_expand_key(bits, key, enc, dec), "aes_expand_key");
    host = read_file(in_path, &len);
    if (!host) return 2;
    nblocks = len / 16;
    if (cudaMalloc((void **)&dev, nblocks * 16 + 16) != cudaSuccess) return 3;
    if (cudaMemcpy(dev, host, nblocks * 16, cudaMemcpyHostToDevice) != cudaSuccess) return 3;
    check(aes_ecb_encrypt(enc, nr, dev, dev, nblocks, NULL), "aes_ecb_encrypt");       /* in place */
    if (cudaMemcpy(host, dev, nblocks * 16, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    if (write_file(enc_path, host, nblocks * 16) != 0) return 2;
    check(aes_ecb_decrypt(dec, nr, dev, dev, nblocks, NULL), "aes_ecb_decrypt");
    if (cudaMemcpy(host, dev, nblocks * 16, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    if (write_file(dec_path, host, nblocks * 16) != 0) return 2;
    cudaFree(dev);
    free(host);
    return 0;
}

int main(int argc, char **argv) {
    if (argc == 3 && strcmp(argv[1], "keys") == 0) return cmd_keys(argv[2]);
    if (argc == 2 && strcmp(argv[1], "errors") == 0) return cmd_errors();
    if (argc == 6 && strcmp(argv[1], "ecb") == 0) return cmd_ecb(argv[2], argv[3], argv[4], argv[5]);
    fprintf(stderr, "usage: aes_client keys <hexkey> | errors | ecb <hexkey> <in> <enc> <dec>\n");
    return 2;
}
