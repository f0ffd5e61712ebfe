/*
 * aesgb.h -- C ABI of the GB300 (sm_103a) bulk AES library.
 *
 * The library implements the method of "GPU Accelerated AES Algorithm"
 * (Wang & Chu, arXiv 1902.05234): AES in Electronic Codebook mode (section
 * 3.1.1, eq (1): C_i = cipher(P_i), every 16-byte block independent), each
 * round folded into four T-table lookups per column (section 3.2.3, eqs
 * (22)-(26)).  Decryption, which the paper reports (Table 5) but does not
 * describe, is the FIPS-197 5.3.5 equivalent inverse cipher with the
 * analogous inverse tables.
 *
 * Conventions for every entry point:
 *  - Return value: AES_OK (0) or a negative aes_status; aes_status_str()
 *    names it.  No entry point aborts, traps or throws.
 *  - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  GPU work is enqueued asynchronously on it; the call neither
 *    allocates device memory nor synchronises (except where stated).  Errors
 *    of the launch itself return AES_E_CUDA; faults during execution surface
 *    at the caller's next synchronisation.
 *  - Data pointers marked DEVICE must point to device memory of the current
 *    device (cudaSetDevice) and stay valid until the enqueued work completes.
 *    Pointers marked HOST are read during the call only.
 *  - Blocks are whole 16-byte AES states; byte i of a block is state entry
 *    s[i mod 4][i / 4] (FIPS-197 3.4).  There is no padding: callers pass a
 *    block count.
 *  - Round keys are the FIPS-197 expanded key as a byte string: word i of
 *    rk holds bytes 4i..4i+3 of that string in memory order, so the layout is
 *    the same on any host.
 *  - CUDA graphs: the first launch of a kernel configuration on a device sets
 *    the kernel's shared-memory limit and caches its occupancy (host calls,
 *    not stream work).  Make one call of each configuration before capturing
 *    the enqueuing calls into a graph; after that they only enqueue kernels.
 *    aes_batch_graph_create does this set-up itself.  aes_ecb_batch and
 *    aes_ecb_batch_ex refuse a capturing stream (their workspace belongs to
 *    the library); capture aes_ecb_batch_ws instead.
 *  - Launch overlap: the single-buffer kernels are launched with
 *    programmatic stream serialisation, so one may start (fill its tables)
 *    while the previous kernel in the stream drains; it waits for that
 *    kernel to complete before touching global memory, so stream order
 *    semantics are unchanged.
 *  - Thread safety: calls may come from several host threads on distinct
 *    streams; library state (caches, tuned configurations, internal streams,
 *    the per-stream batch workspaces) is guarded.  A server handle is the
 *    exception (see aes_srv_create).
 */
#ifndef AESGB_H
#define AESGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* Status codes                                                              */
/* ------------------------------------------------------------------------ */
typedef enum aes_status {
    AES_OK = 0,
    AES_E_ARG = -1,      /* null pointer, size overflow or bad enum value      */
    AES_E_KEYBITS = -2,  /* key size not 128, 192 or 256 bits                  */
    AES_E_NROUNDS = -3,  /* nrounds not 10, 12 or 14                           */
    AES_E_ALIGN = -4,    /* a block pointer not 16-byte aligned                */
    AES_E_OVERLAP = -5,  /* in and out overlap without being equal             */
    AES_E_CUDA = -6,     /* a CUDA runtime call failed (launch, attribute ...) */
    AES_E_NOMEM = -7,    /* an allocation the call documents failed            */
    AES_E_TIMEOUT = -8,  /* a bounded wait ran out                             */
    AES_E_BUSY = -9,     /* admission refused: budget or slots full            */
    AES_E_RANGE = -10,   /* a size above a documented maximum                  */
    AES_E_NOTFOUND = -11,/* unknown key id or ticket                           */
    AES_E_CONFIG = -12,  /* launch configuration not supported                 */
    AES_E_CANCELLED = -13,   /* a server request cancelled before its launch   */
    AES_E_UNREGISTERED = -14 /* a server buffer outside every registered range */
} aes_status;

/* Name of a status code (static string; "unknown status" for other values). */
const char *aes_status_str(int status);

/* Library version, major*10000 + minor*100 + patch. */
int aes_version(void);

/* Number of bounded device-side waits (the TMA-staged kernel's mbarrier
 * waits, about one second each) that ran out since the last call, summed
 * over all launches on the current device; reading resets it.  A timed-out
 * warp stops without finishing its blocks, so a non-zero count means some
 * output of those launches is missing.  DEVICE-synchronous (a cudaMemcpy
 * from the counter). */
int aes_wait_timeouts(unsigned long long *count);

/* Debug build only (libaesgb_debug.so, compiled with AESGB_BOUNDS_CHECK):
 * the number of index checks that failed in any kernel since the last call,
 * summed over the kernels' translation units; reading resets it.  The debug
 * build checks every shared-memory table, tile, mask and key-slot access and
 * the global ranges the batch and TMA kernels derive on the device; a failed
 * check is counted and its access skipped (nothing traps).  AES_E_CONFIG with
 * *count = 0 in the release build.  DEVICE-synchronous. */
int aes_debug_bounds_violations(unsigned long long *count);

/* Failure-injection test hook (host side, every build).  Of the memory
 * allocations the library makes for itself from now on -- the device and
 * page-locked host memory of aes_srv_create, the library-owned batch
 * workspace of aes_ecb_batch -- the first `skip` succeed and the `count`
 * after them fail as if the device were out of memory, so that each caller's
 * AES_E_NOMEM path and its clean-up run without a real shortage.  count = 0
 * disarms it.  AES_E_ARG if either is negative.  Process-wide. */
int aes_test_fail_allocs(int skip, int count);

/* Debug build only: exactly-once coverage of the batch kernel's work counter.
 * Each chunk (chunk_blocks consecutive blocks of one message, the unit a warp
 * takes from the counter) adds one to its tag, for chunk indices below 65,536.
 * Returns, over all batch launches since the last call: *once the chunks
 * tagged exactly once, *repeated those tagged more than once, *beyond the
 * chunks whose index lies past the tags; then clears the tags.  After ONE
 * launch of T <= 65,536 chunks, *once == T and the others are 0.
 * AES_E_CONFIG with all three 0 in the release build.  DEVICE-synchronous. */
int aes_debug_batch_coverage(unsigned long long *once, unsigned long long *repeated, unsigned long long *beyond);

/* Failure-detection test hook: one warp of the TMA-staged encryption kernel
 * on nblocks (1..64) DEVICE blocks, with every mbarrier expecting 16 bytes
 * more than its bulk copy delivers.  The copies land, but no wait can finish:
 * each runs out after about one second, the warp counts one timeout (read
 * with aes_wait_timeouts), waits (bounded) for its copies and stops without
 * writing `out`.  The context stays usable.  Async on `stream`; the kernel
 * takes about 1-3 s.  AES_E_RANGE outside 1..64 blocks, AES_E_ALIGN /
 * AES_E_OVERLAP as aes_ecb_encrypt. */
int aes_tma_selftest_timeout(const uint8_t *in, uint8_t *out, size_t nblocks, void *stream);

/* ------------------------------------------------------------------------ */
/* Key schedule (host)                                                       */
/* ------------------------------------------------------------------------ */

/* Expand a cipher key into round keys.  Paper section 3.2.2 (key expansion
 * and round-key selection, Nr+1 round keys of 128 bits) and Algorithm 1
 * step 1; the steps (RotWord, SubWord, Rcon) follow FIPS-197 5.2.
 *   keybits  128, 192 or 256; key: HOST, keybits/8 bytes.
 *   rk_enc   HOST, caller-owned, at least 4*(Nr+1) words (60 always suffice):
 *            the expanded key w[0 .. 4*Nr+3].  May be NULL.
 *   rk_dec   HOST, same size: the equivalent-inverse-cipher schedule dw of
 *            FIPS-197 5.3.5 (w with InvMixColumns applied to round keys
 *            1..Nr-1), in the same word order as w.  May be NULL.
 * Returns Nr (10, 12 or 14) on success, AES_E_KEYBITS or AES_E_ARG.
 * Host only: touches no GPU. */
int aes_expand_key(int keybits, const uint8_t *key, uint32_t *rk_enc, uint32_t *rk_dec);

/* ------------------------------------------------------------------------ */
/* Single-buffer ECB                                                         */
/* ------------------------------------------------------------------------ */

/* ECB encryption of nblocks independent 16-byte blocks, eq (1), each block
 * run through the initial AddRoundKey, Nr-1 T-table rounds (eq (26)) and the
 * final round without MixColumns (FIPS-197 5.1; Algorithm 1 as printed is
 * wrong there).
 *   rk       HOST, 4*(nrounds+1) words from aes_expand_key (rk_enc).  Copied
 *            into the launch parameters: it may be freed on return.
 *   nrounds  10, 12 or 14.
 *   in, out  DEVICE, 16-byte aligned, nblocks*16 bytes each.  in == out
 *            (in place) is allowed; any other overlap is AES_E_OVERLAP.
 *   nblocks  0 is a no-op returning AES_OK.
 * Launch configuration: the tuned configuration for (direction, nrounds,
 * size) if one was recorded with aes_tune*, else the built-in default. */
int aes_ecb_encrypt(const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out,
                    size_t nblocks, void *stream);

/* ECB decryption, the same contract with rk_dec from aes_expand_key: the
 * FIPS-197 5.3.5 equivalent inverse cipher (T-table form with the inverse
 * tables, InvS in the final round). */
int aes_ecb_decrypt(const uint32_t *rk_dec, int nrounds, const uint8_t *in, uint8_t *out,
                    size_t nblocks, void *stream);

/* Placement of the lookup tables (the paper's design axis of section 4.2). */
typedef enum aes_layout {
    AES_LAYOUT_R4 = 0,    /* 4 tables in shared memory, one copy per bank: 128 KiB
                             (enc) / 160 KiB (dec); conflict-free, 1 CTA per SM   */
    AES_LAYOUT_R1 = 1,    /* 1 table per bank-replicated + byte rotations: 64 KiB  */
    AES_LAYOUT_P4 = 2,    /* 4 plain 1 KiB tables in shared memory (bank conflicts) */
    AES_LAYOUT_CONST = 3, /* tables in constant memory, as in the paper (4.2)      */
    AES_LAYOUT_R4_TMA = 4,/* (plaintext placement, section 4.4) R4 tables; the
                             plaintext staged into shared memory by
                             TMA bulk copies (two 512 x blocks_per_thread-byte
                             tiles per warp, mbarrier-tracked, two passes ahead)
                             instead of loaded into registers                     */
    AES_LAYOUT_R2 = 5,    /* tables 0 and 1 bank-replicated: 64 KiB (enc) /
                             128 KiB (dec); tables 2 and 3 are their 16-bit
                             rotations, applied once per column to the XOR of
                             the pair's two lookups (eqs (22)-(25): T_k is T_0
                             rotated by k bytes)                                  */
    AES_LAYOUT_REG = 6    /* the table in registers (section 4.2's third
                             placement): each warp's 32 lanes hold the 256
                             entries of T0, eight each; a lookup gathers the
                             eight candidates from one lane by warp shuffles
                             and selects one; T1..T3 by byte rotation.  No
                             shared memory; blocks_per_thread 1 or 2, at
                             most 256 threads                                  */
} aes_layout;

/* A launch configuration of the ECB kernels. */
typedef struct aes_launch_cfg {
    int32_t threads;           /* threads per CTA, multiple of 32, 32..1024
                                  (<= 512 when blocks_per_thread is 4, <= 256
                                  when it is 8)                                 */
    int32_t blocks_per_thread; /* AES blocks per thread per pass: 1, 2, 4 or 8
                                  (granularity 16, 32, 64 or 128 bytes per
                                  thread; 8 with layouts R4 and R2 only)        */
    int32_t layout;            /* aes_layout                                     */
    int32_t ctas_per_sm;       /* persistent grid = ctas_per_sm x SM count;
                                  0 = as many as fit                             */
} aes_launch_cfg;

/* ECB with an explicit launch configuration (the autotuner and the
 * placement study use it).  dir 0 = encrypt with rk_enc, 1 = decrypt with
 * rk_dec; otherwise as aes_ecb_encrypt.  AES_E_CONFIG for an unsupported
 * combination. */
int aes_ecb_crypt_cfg(int dir, const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out,
                      size_t nblocks, const aes_launch_cfg *cfg, void *stream);

/* The configuration aes_ecb_encrypt/decrypt would use for this call. */
int aes_ecb_get_cfg(int dir, int nrounds, size_t nblocks, aes_launch_cfg *cfg);

/* ------------------------------------------------------------------------ */
/* Batched ECB: many messages, one persistent launch                         */
/* ------------------------------------------------------------------------ */

/* One message of a batch: ECB (eq (1)) over nblocks blocks with its own key,
 * key size and direction.  The descriptor table lives in DEVICE memory.
 *   rk       DEVICE, 4*(nrounds+1) words: rk_enc for dir 0, rk_dec (FIPS dw
 *            order, exactly as aes_expand_key writes it) for dir 1.
 *   in, out  DEVICE, 16-byte aligned; equal or disjoint.  Outputs of different
 *            messages must not overlap each other or any input.
 *   nblocks  may be 0 (nothing to do).
 *   nrounds  10, 12 or 14.   dir  0 encrypt, 1 decrypt.
 * A descriptor that breaks these rules is skipped (its output untouched) and
 * its status (AES_E_NROUNDS, AES_E_ARG, AES_E_ALIGN, AES_E_OVERLAP) is written
 * to the optional status array; the other messages are processed. */
typedef struct aes_desc {
    const uint32_t *rk;
    const uint8_t *in;
    uint8_t *out;
    uint64_t nblocks;
    int32_t nrounds;
    int32_t dir;
} aes_desc;

/* Launch configuration of the batch kernel (tables always bank-replicated). */
typedef struct aes_batch_cfg {
    int32_t threads;           /* threads per CTA (multiple of 32, <= 512: keys sit in registers)    */
    int32_t blocks_per_thread; /* 1, 2 or 4                                                           */
    int32_t chunk_passes;      /* a warp's unit of work = 32 * blocks_per_thread * chunk_passes blocks */
    int32_t ctas_per_sm;       /* 0 or 1 (the tables take most of the shared memory)                */
    int32_t layout_enc;        /* table layout of the encryption phase and of the decryption      */
    int32_t layout_dec;        /* phase (aes_layout; section 4.2): the pairs R4/R2 (the default,
                                  blocks_per_thread 1, 2 or 4), R4/R4, R2/R2 and R1/R1 (1 or 2);
                                  another pair is AES_E_CONFIG                                       */
} aes_batch_cfg;

/* Bytes of DEVICE workspace a batch of n descriptors needs (plan header, the
 * message order and the chunk prefix: about 20 bytes per descriptor). */
size_t aes_batch_workspace_bytes(int n);

/* Most descriptors one batch call takes (AES_E_RANGE above it, nothing queued). */
#define AES_BATCH_MAX_DESCS (1 << 28)

/* Batched ECB with a caller-owned workspace.  Enqueues two kernels on
 * `stream`: a one-CTA plan kernel (validation, encryptions-first order, chunk
 * prefix) and the persistent batch kernel (one CTA per SM; each warp takes
 * the next chunk from an atomic work counter, finds the chunk's message by a
 * warp-wide 32-ary search of the prefix and stages its round keys through
 * shared memory into registers).  Allocates nothing and never synchronises,
 * so it can be captured in a CUDA graph.
 *   n           0..AES_BATCH_MAX_DESCS.
 *   desc_dev    DEVICE array of n descriptors, unchanged until completion.
 *   ws          DEVICE, 256-byte aligned, ws_bytes >= aes_batch_workspace_bytes(n);
 *               owned by the caller and busy until completion.
 *   status_dev  DEVICE int32[n] or NULL: per-message aes_status.
 *   cfg         NULL for the tuned/default configuration.
 * Returns AES_E_RANGE if ws is too small, AES_E_CONFIG for a bad cfg. */
int aes_ecb_batch_ws(const aes_desc *desc_dev, int n, void *ws, size_t ws_bytes, int32_t *status_dev,
                     const aes_batch_cfg *cfg, void *stream);

/* Batched ECB with a library-owned workspace: the same as aes_ecb_batch_ws
 * (default configuration, no status array) with a workspace the library keeps
 * per (device, stream) -- streams told apart by their CUDA stream id, so each
 * host thread's per-thread default stream has its own.  The workspace is
 * allocated on the first call on a stream (at least 1 MiB) and grown when n
 * needs more.  Allocation and growth are stream-ordered (cudaMallocAsync /
 * cudaFreeAsync on `stream`): the call never synchronises the device nor
 * waits for other streams, and the buffer it replaces is released only after
 * the batches already queued on `stream`.  Calls may come from several host
 * threads at once, on the same or on different streams; calls on different
 * streams never share a workspace.  Workspaces are freed by aes_shutdown; once
 * more than 64 exist, the idle ones (last batch complete) of other streams are
 * released when a new stream makes one.
 *   desc_dev  DEVICE array of n descriptors (NULL with n > 0: AES_E_ARG).
 * AES_E_NOMEM if the workspace cannot be allocated (nothing is enqueued, the
 * stream's old workspace stays).  A stream that is being captured into a CUDA
 * graph is refused with AES_E_CONFIG, nothing enqueued: the graph would keep
 * the address of a workspace that a later call on the stream may release --
 * capture aes_ecb_batch_ws with a caller-owned workspace instead. */
int aes_ecb_batch(const aes_desc *desc_dev, int n, void *stream);

/* Batched ECB that allocates nothing: not even the workspace.  The paper has
 * no counterpart; this exists for callers that must not allocate device
 * memory -- for example a plugin whose host application hands out only the
 * buffers it owns, code that runs while another thread is capturing a CUDA
 * graph in global mode (cudaMalloc is refused then), or a serving thread that
 * cannot afford cudaMalloc/cudaFree synchronising the whole device.
 * Same contract and work as aes_ecb_batch_ws, except that the workspace is a
 * fixed array in the library's device memory (about 330 KB per device that
 * loads the library, held until the process exits):
 *   n  at most AES_BATCH_NOALLOC_MAX_DESCS, else AES_E_RANGE (nothing queued).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and sets the batch kernel's shared-memory
 * limit; make that first call before any stream capture.  While another
 * thread captures in global mode, call it on a stream created with
 * cudaStreamNonBlocking: work on the legacy default stream (stream NULL) is
 * refused then and invalidates that capture.  Every call on a device uses the
 * same array, so calls whose work overlaps on the GPU (different streams
 * without ordering) race and corrupt each other: order them on one stream or
 * synchronise between them. */
/* aes_ecb_batch with the optional per-message status array of
 * aes_ecb_batch_ws (status_dev: DEVICE int32[n] or NULL), i.e. the library
 * workspace per (device, stream) and the default or tuned configuration. */
int aes_ecb_batch_ex(const aes_desc *desc_dev, int n, int32_t *status_dev, void *stream);

#define AES_BATCH_NOALLOC_MAX_DESCS 16384
int aes_ecb_batch_noalloc(const aes_desc *desc_dev, int n, int32_t *status_dev, void *stream);

/* A batch captured once as a CUDA graph (plan + batch kernel) and replayed.
 * desc_dev, ws and status_dev are baked in; the CONTENTS of the descriptor
 * table may change between launches (the plan kernel reads it at run time),
 * n may not.  aes_batch_graph_launch enqueues one replay on `stream`. */
typedef struct aes_batch_graph aes_batch_graph;
int aes_batch_graph_create(const aes_desc *desc_dev, int n, void *ws, size_t ws_bytes, int32_t *status_dev,
                           const aes_batch_cfg *cfg, aes_batch_graph **graph);
int aes_batch_graph_launch(aes_batch_graph *graph, void *stream);
int aes_batch_graph_destroy(aes_batch_graph *graph);

/* ECB over HOST buffers: the path a caller takes whose data is in host
 * memory.  Same cipher as aes_ecb_encrypt/decrypt (dir 0 = encrypt with
 * rk_enc, 1 = decrypt with rk_dec; rk HOST, copied during the call).
 *   host_in, host_out  HOST, nblocks*16 bytes; equal (in place) or disjoint.
 *                      Page-locked memory (cudaHostAlloc / cudaHostRegister)
 *                      lets the copies overlap the kernels; pageable memory
 *                      works but the copies then serialise.
 *   dev_buf            DEVICE staging buffer, caller-owned, 16-byte aligned,
 *                      dev_buf_bytes >= 48; it is split into 3 slots and the
 *                      data moves through it in chunks of dev_buf_bytes/3.
 * The chunks are copied in, ciphered in place and copied out on three
 * streams the library creates on the first call per device (released by
 * aes_shutdown), so copies and kernels of successive chunks overlap.  The
 * call is asynchronous: `stream` first waits for its earlier work, then is
 * made to wait for the last copy-out, so synchronising `stream` means the
 * result is in host_out.  Host buffers and dev_buf must stay valid until
 * then.  Calls on one device are serialised on the internal streams. */
int aes_ecb_host(int dir, const uint32_t *rk, int nrounds, const uint8_t *host_in,
                 uint8_t *host_out, size_t nblocks, uint8_t *dev_buf, size_t dev_buf_bytes,
                 void *stream);

/* ECB directly on page-locked HOST memory: host_in and host_out must be
 * page-locked and mapped for the device (cudaHostAlloc / cudaHostRegister with
 * mapping, or torch's pin_memory), else AES_E_ARG.  The kernel reads and
 * writes them over the host link itself -- no staging buffer, no copies, no
 * internal streams; throughput is that of the link.  Same cipher, rk and
 * overlap rules as aes_ecb_encrypt/decrypt; asynchronous on `stream`.  The
 * buffers must hold nblocks*16 bytes (only their first bytes are checked). */
int aes_ecb_host_direct(int dir, const uint32_t *rk, int nrounds, const uint8_t *host_in, uint8_t *host_out,
                        size_t nblocks, void *stream);

/* ------------------------------------------------------------------------ */
/* Other parallel modes on the same cipher                                   */
/* ------------------------------------------------------------------------ */

/* CTR (section 3.1.5, eq (5); Table 1: parallel like ECB): C_i = P_i xor
 * E(T_i) with T_i = ctr0 + i as a 128-bit big-endian integer mod 2^128 (ctr0,
 * HOST, 16 bytes, is the counter block of the first block).  The same call
 * decrypts.  rk = rk_enc (HOST); in/out DEVICE as for ECB, in place allowed. */
int aes_ctr_crypt(const uint32_t *rk, int nrounds, const uint8_t *ctr0, const uint8_t *in, uint8_t *out,
                  size_t nblocks, void *stream);

/* CBC decryption (section 3.1.2, with eq (2) read as C_i = E(P_i xor C_{i-1})
 * per NIST SP 800-38A): P_i = D(C_i) xor C_{i-1}, C_{-1} = iv (HOST, 16 bytes).
 * Every block needs only two ciphertext blocks, so it runs in parallel.
 * rk_dec from aes_expand_key; in/out DEVICE, disjoint (in place is
 * AES_E_OVERLAP: ciphertext must outlive the plaintext written next to it).
 * CBC encryption chains block to block and is not offered (Table 1). */
int aes_cbc_decrypt(const uint32_t *rk_dec, int nrounds, const uint8_t *iv, const uint8_t *in, uint8_t *out,
                    size_t nblocks, void *stream);

/* CFB decryption (section 3.1.3, with eq (3) read as its text states --
 * the mode is fed with the previous ciphertext -- i.e. full-block CFB of
 * NIST SP 800-38A: C_i = P_i xor E(C_{i-1}), C_{-1} = iv): P_i = C_i xor
 * E(C_{i-1}), the FORWARD cipher, so rk = rk_enc from aes_expand_key.  Every
 * block needs only two ciphertext blocks, so it runs in parallel.  iv HOST,
 * 16 bytes; in/out DEVICE, disjoint (in place is AES_E_OVERLAP, as for CBC).
 * CFB encryption chains block to block and is not offered (Table 1). */
int aes_cfb_decrypt(const uint32_t *rk_enc, int nrounds, const uint8_t *iv, const uint8_t *in, uint8_t *out,
                    size_t nblocks, void *stream);

/* Release every resource the library created lazily on all devices: the
 * host pipeline's internal streams and events and the library-owned batch
 * workspaces.  Call with no work of the library in flight.  Later calls
 * create them again as needed.  Tuned configurations stay (aes_tune_clear
 * drops them); the fixed scratch of aes_ecb_batch_noalloc lives until exit. */
int aes_shutdown(void);

/* ------------------------------------------------------------------------ */
/* Constant-time ECB (bitsliced)                                             */
/* ------------------------------------------------------------------------ */
/* ECB without table lookups, for callers that need the cipher to be free of
 * data- and key-dependent memory accesses (the side channel behind the
 * paper's remark on xtime and power analysis, section 3.2.1).  Each thread
 * transposes 32 blocks into 128 bit planes and runs every round as fixed
 * circuits of 3-input logic gates: a tower-field GF((2^4)^2) inversion
 * circuit with the affine map for SubBytes, a register permutation for
 * ShiftRows, a MixColumns circuit (decryption: one circuit per column for
 * the inverse S-box's output map and InvMixColumns); round keys enter the
 * S-box circuits as mask planes.  Same results and the same contract as
 * aes_ecb_crypt_cfg: dir 0 encrypt with rk_enc, 1 decrypt with rk_dec
 * (HOST); in/out DEVICE, 16-byte aligned, equal or disjoint. */
int aes_ecb_crypt_ct(int dir, const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out, size_t nblocks,
                     void *stream);

/* Logic operations (one 3-input gate or byte permute each, the integer-logic
 * pipe's unit of work) that aes_ecb_crypt_ct spends per 16-byte block for
 * direction dir and nrounds rounds, counted from its circuits: the key of
 * step 0 on the planes, the rounds' S-box, MixColumns / InvMixColumns and
 * output circuits, and the two in-register 32x32 transposes per column
 * (their shifts run on the multiply pipe and are not counted).  Host only;
 * *ops_per_block written on AES_OK; bad dir / nrounds / NULL -> AES_E_ARG /
 * AES_E_NROUNDS. */
int aes_ct_ops_per_block(int dir, int nrounds, double *ops_per_block);

/* Test hook: the same bitsliced code run on the host over HOST buffers, so
 * the circuit can be checked against a reference without a GPU.  Not used by
 * any other entry point. */
int aes_ct_selftest_host(int dir, const uint32_t *rk, int nrounds, const uint8_t *in, uint8_t *out,
                         size_t nblocks);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching over the batch kernel                        */
/* ------------------------------------------------------------------------ */
/* A request is ECB (eq (1)) of one caller-owned device buffer with a
 * resident key.  The server's dispatcher thread admits requests in arrival
 * order while the bytes in flight (2 x nbytes per admitted, unfinished
 * request: input and output) stay within mem_budget_bytes, packs what is
 * admitted -- at most mem_budget_bytes / slots per batch, so that several
 * batches queue on the device under load -- into one batch whenever one of
 * `slots` in-flight batch slots is free, plans it on the host (requests are
 * validated at submission) and launches it on that slot's stream (descriptor
 * and plan upload, the persistent batch kernel, completion event).  Requests
 * that arrive while earlier batches run join the next batch; consecutive
 * batches overlap on the device.  With device timing on
 * (aes_srv_set_device_timing), a batch's device interval runs from the moment
 * its stream reaches the kernel (descriptors uploaded; a timing event) to the
 * kernel's completion (another); aes_srv_stats then reports how many such
 * intervals overlapped at most, and for how long.  The dispatcher holds the
 * server's lock only to pack and to retire batches, never across CUDA calls.
 * Host waits are bounded; nothing waits on the device.  Latency = host
 * arrival -> host-observed completion.
 * A server handle is used from one host thread at a time (plus its own
 * dispatcher); it works on the device that was current at creation. */
typedef struct aes_server aes_server;

typedef struct aes_srv_stats_t {
    uint64_t submitted, completed, batches, bytes_completed;
    uint64_t inflight_bytes, peak_inflight_bytes, pending;
    double busy_s;          /* first arrival -> last completion            */
    int32_t worker_status;  /* AES_OK, or the first dispatcher CUDA error   */
    int32_t reserved;
    uint64_t cancelled;     /* requests completed by aes_srv_cancel         */
    uint64_t peak_busy_slots;     /* most slots holding a launched, not yet
                                     retired batch at once (host view)       */
    uint64_t timed_batches;       /* batches whose device interval was taken
                                     (device timing on)                       */
    uint64_t peak_device_batches; /* most batches whose device intervals
                                     contain one instant                      */
    double device_overlap_s;      /* time in which two or more batches'
                                     device intervals overlap                 */
} aes_srv_stats_t;

/* Create a server: key store for max_keys expanded schedules (device),
 * `slots` in-flight batches (1..16), at most max_batch requests per batch
 * (1..AES_BATCH_MAX_DESCS, else AES_E_RANGE).  Allocates its device and
 * page-locked memory here (AES_E_NOMEM). */
int aes_srv_create(size_t mem_budget_bytes, int max_keys, int max_batch, int slots, aes_server **srv);

/* Expand key (HOST, keybits/8 bytes) and keep both schedules resident under
 * key_id (0..max_keys-1).  The upload runs on a stream of the server's own,
 * and every batch launched afterwards waits for it on the device; the call
 * returns once the bytes are staged, without waiting for the device.
 * Replacing a key that a queued or in-flight request names is refused with
 * AES_E_BUSY (the request would otherwise run with the new key): drain or
 * cancel those requests first.  While the upload is being issued, submissions
 * naming key_id answer AES_E_BUSY.  AES_E_CUDA if the upload fails. */
int aes_srv_put_key(aes_server *srv, int key_id, int keybits, const uint8_t *key);

/* The same with the key already expanded: rk_enc and rk_dec (HOST,
 * 4*(nrounds+1) words each, as aes_expand_key writes them), nrounds 10, 12 or
 * 14 (AES_E_NROUNDS).  Same upload, refusal and ordering as aes_srv_put_key. */
int aes_srv_put_schedule(aes_server *srv, int key_id, const uint32_t *rk_enc, const uint32_t *rk_dec,
                         int nrounds);

/* Submit one request arriving now: in_dev/out_dev DEVICE, 16-byte aligned,
 * equal or disjoint, nbytes a multiple of 16 with 2*nbytes <= budget
 * (AES_E_RANGE), key_id resident (AES_E_NOTFOUND; AES_E_BUSY while
 * aes_srv_put_key is uploading it).  *ticket identifies it. */
int aes_srv_submit(aes_server *srv, int key_id, int dir, const uint8_t *in_dev, uint8_t *out_dev,
                   size_t nbytes, uint64_t *ticket);

/* Submit n requests whose arrival times are now + arrival_offsets_s[i]
 * (seconds, non-decreasing; NULL = all now) -- an open-loop request stream
 * replayed by the server.  Arrays are HOST; device addresses as uint64.
 * tickets[i] = 0 for a rejected request; returns the first rejection status. */
int aes_srv_submit_many(aes_server *srv, int n, const int32_t *key_ids, const int32_t *dirs,
                        const uint64_t *in_devs, const uint64_t *out_devs, const uint64_t *nbytes,
                        const double *arrival_offsets_s, uint64_t *tickets);

/* Non-blocking check: *done = 1 once finished; then *status (per-request
 * aes_status) and *latency_s (may be NULL). */
int aes_srv_poll(aes_server *srv, uint64_t ticket, int *done, int *status, double *latency_s);

/* Block up to timeout_ms for one request (AES_E_TIMEOUT), or for all (drain). */
int aes_srv_wait(aes_server *srv, uint64_t ticket, int timeout_ms, int *status, double *latency_s);
int aes_srv_drain(aes_server *srv, int timeout_ms);

/* Statuses, latencies and queueing delays (arrival -> admission) of n
 * finished requests (HOST arrays, any may be NULL except tickets); release != 0
 * forgets them afterwards.  AES_E_BUSY if some are not finished. */
int aes_srv_results(aes_server *srv, int n, const uint64_t *tickets, int32_t *status, double *latency_s,
                    double *queue_s, int release);

int aes_srv_stats(aes_server *srv, aes_srv_stats_t *out);

/* Device timing of batches, off by default: on != 0 records two timing events
 * per batch from the next busy period (the next launch that finds every slot
 * idle) on, so that aes_srv_stats reports timed_batches, peak_device_batches
 * and device_overlap_s; 0 stops it from the next busy period on.  The events
 * add about 10 us to a light-load request's latency (measured on GB300), so
 * leave it off where latency matters.  Host-side counters (peak_busy_slots,
 * peak_inflight_bytes) are kept either way. */
int aes_srv_set_device_timing(aes_server *srv, int on);

/* Cancel a request that has not been launched yet (still queued: not arrived,
 * or waiting for budget or a slot).  It completes at once with status
 * AES_E_CANCELLED, its buffers are never touched, and aes_srv_drain no longer
 * waits for it.  AES_E_BUSY if the request is already in a launched batch or
 * done (it then completes, or has completed, normally); AES_E_NOTFOUND for an
 * unknown or released ticket. */
int aes_srv_cancel(aes_server *srv, uint64_t ticket);

/* Registry of the device allocations requests may use.  While it is empty
 * (the default) every buffer is accepted.  Once a range is registered,
 * aes_srv_submit* accept a request only if its input and its output each lie
 * entirely inside one registered range, and return AES_E_UNREGISTERED
 * otherwise -- a host-side check before anything is launched, so that a
 * descriptor can never point outside the caller's allocations.  Ranges may
 * not overlap (AES_E_OVERLAP); unregistering (AES_E_NOTFOUND for an unknown
 * base) affects later submissions only. */
int aes_srv_register(aes_server *srv, const void *base_dev, size_t bytes);
int aes_srv_unregister(aes_server *srv, const void *base_dev);

/* Stop the dispatcher (requests not yet launched are dropped), wait for the
 * batches in flight and free everything. */
int aes_srv_destroy(aes_server *srv);

/* ------------------------------------------------------------------------ */
/* Autotuner                                                                 */
/* ------------------------------------------------------------------------ */
/* The granularity (16, 32 or 64 bytes per thread: the axis of the paper's
 * related work, section 2) and the table placement (section 4.2) are chosen
 * per GPU by timing.  Tuned entries are kept per (SM count, direction,
 * nrounds, size class = floor(log4(nblocks))) for the single-buffer calls and
 * per SM count for batches; aes_ecb_encrypt/decrypt and the batch calls use
 * them from then on.  If the environment variable AESGB_TUNE_CACHE names a
 * file, entries are loaded from it on first use and written to it after each
 * tuning run.  Tuning launches the kernels many times on the given buffers
 * (out is overwritten, in is only read): each candidate is captured in a CUDA
 * graph of back-to-back launches on a stream of the tuner's own, which first
 * waits for `stream`, and the replay is timed on the device.  The call
 * synchronises that stream, makes `stream` wait for it and takes seconds. */

/* Tune the single-buffer kernel for (dir, nrounds, size class of nblocks) on
 * the caller's DEVICE buffers (same rules as aes_ecb_crypt_cfg; rk HOST).
 * best (HOST, may be NULL) receives the chosen configuration. */
int aes_tune_ecb(int dir, int nrounds, const uint32_t *rk, const uint8_t *in, uint8_t *out, size_t nblocks,
                 void *stream, aes_launch_cfg *best);

/* Tune the batch kernel on a caller's batch (same arguments as
 * aes_ecb_batch_ws without status; the batch is run many times). */
int aes_tune_batch(const aes_desc *desc_dev, int n, void *ws, size_t ws_bytes, void *stream,
                   aes_batch_cfg *best);

/* Tune the single-buffer kernel for (dir, nrounds, size class of
 * bytes_hint / 16 blocks) without caller buffers: the call allocates an input
 * and an output of bytes_hint bytes (stream-ordered on `stream`, released at
 * the end; AES_E_NOMEM if they cannot be had) and runs aes_tune_ecb on them
 * with an all-zero key (the kernels' time does not depend on key or data).
 * AES_E_ARG for bytes_hint below 16. */
int aes_tune(int dir, int nrounds, size_t bytes_hint, void *stream);

/* Record a configuration by hand for (dir, nrounds, size class of nblocks). */
int aes_tune_set_ecb(int dir, int nrounds, size_t nblocks, const aes_launch_cfg *cfg);

/* The configuration the batch calls would use for n descriptors. */
int aes_batch_get_cfg(int n, aes_batch_cfg *cfg);

/* Write / read the tuned entries to / from a text file (path HOST); clear all
 * entries (the defaults apply again). */
int aes_tune_save(const char *path);
int aes_tune_load(const char *path);
int aes_tune_clear(void);

/* ------------------------------------------------------------------------ */
/* Introspection                                                             */
/* ------------------------------------------------------------------------ */

/* Number of SMs of CUDA device `device` (>0), or AES_E_CUDA. */
int aes_device_sm_count(int device);

/* Measure the sustainable rate of the bound the T-table kernels run into:
 * independent, bank-conflict-free 4-byte shared-memory lookups (the access
 * pattern of eq (26) without the rest of the cipher), one CTA of 1,024 threads
 * per SM.  sink_dev: DEVICE scratch of at least SMs*4096 bytes (only written
 * in a case that does not occur; it keeps the loads from being removed).
 * Returns the lookups performed and the seconds they took (synchronises
 * `stream`); lookups / seconds / (SMs * SM clock) is the measured peak per
 * SM per clock, against the nominal 32. */
int aes_calibrate_lookup_rate(void *sink_dev, size_t sink_bytes, void *stream, double *lookups, double *seconds);

/* The same for the bound of the constant-time kernel: three-input logic
 * instructions (LOP3), eight independent chains per thread, one CTA of 1,024
 * threads per SM.  Returns the thread-level operations performed and the
 * seconds they took (synchronises `stream`); ops / seconds / (SMs * SM
 * clock) is the measured peak in lanes per clock per SM, against the nominal
 * 64.  sink_dev as for aes_calibrate_lookup_rate. */
int aes_calibrate_logic_rate(void *sink_dev, size_t sink_bytes, void *stream, double *ops, double *seconds);

/* Copy one of the library's 256-entry tables (built at compile time) from
 * HOST memory, no GPU needed:  which = 0 te0 (eq (22) column packed with row r
 * in byte r), 1 td0 (inverse-cipher column 0e/09/0d/0b * InvS), 2 S-box,
 * 3 inverse S-box (one byte per word).  out: HOST, 256 words. */
int aes_host_table(int which, uint32_t *out);

/* The same tables as the kernels see them in constant memory of the current
 * device (synchronous copy).  out: HOST, 256 words. */
int aes_device_table(int which, uint32_t *out);

#ifdef __cplusplus
}
#endif

#endif /* AESGB_H */
