/*
 * rs_gb300.h - C ABI of the GB300 (sm_103a) Reed-Solomon erasure-coding
 * library: systematic RS(k, m) over GF(2^w), w in {8, 16}, in the
 * polynomial realization of "On the Effectiveness of Polynomial Realization
 * of Reed-Solomon Codes for Storage Systems" (§3), with the Vandermonde and
 * Cauchy bit-matrix matrix realizations (§2) as peers.
 *
 * Conventions shared by every entry point
 *   - Blocks: a stripe is k data blocks d_0..d_{k-1} and m parity blocks
 *     p_0..p_{m-1} of `block_bytes` bytes each.  Block index b in [0, n),
 *     n = k + m: b < k is d_b, b >= k is p_(b-k).  Symbol t of every block
 *     forms one column (one codeword); w = 8 symbols are bytes, w = 16
 *     symbols are little-endian 16-bit words.
 *   - Pointers: every block pointer is a DEVICE pointer, 16-byte aligned,
 *     owned by the caller (with block_bytes = 0 nothing is accessed and any
 *     pointer, NULL included, is accepted).  Pointer arrays are HOST arrays,
 *     read during the call only.  Input and output blocks must not overlap.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Work is enqueued asynchronously; the call returns once it is enqueued.
 *   - Errors: argument errors are detected on the host, return before any
 *     work is enqueued and set a thread-local message (rs_last_error).  A
 *     failed kernel launch returns RS_ECUDA.  Kernel-side timeouts of the
 *     bounded shared-memory pipeline waits are reported through the code's
 *     device status word (rs_poll_status).  No C++ exception crosses the ABI.
 *   - Limits of the device path: n <= 64, m <= 8 (m <= 4 for w = 16),
 *     n <= 2^w - 1.
 */
#ifndef RS_GB300_H
#define RS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rs_code rs_code;
typedef struct rs_batch rs_batch;

typedef enum {
  RS_POLY = 0,           /* generator polynomial g(x) = prod_{i<m}(x + alpha^i), §3 */
  RS_VANDERMONDE = 1,    /* systematic Vandermonde generator matrix, §2.2 */
  RS_CAUCHY = 2,         /* Cauchy generator, bit-matrix XOR over packets, §2.3 */
  RS_POLY_MATRIX = 3,    /* the polynomial code through its generator matrix
                            (column i = x^(m+i) mod g(x), §6); same bytes as RS_POLY */
  RS_POLY_BITMATRIX = 4, /* that matrix's bit-matrix projection over packets
                            (§6 with §2.3's packet layout) */
  RS_GOOD_CAUCHY = 5     /* "good" Cauchy generator (§2.3; GoodCRS of §5.1):
                            the RS_CAUCHY matrix with every column divided by
                            its row-0 entry and every other row divided by the
                            divisor (1 or one of its entries) that leaves the
                            fewest ones; bit-matrix XOR over packets */
} rs_realization;

typedef enum {
  RS_OK = 0,
  RS_EINVAL = 1,             /* bad argument (null, misaligned, bad size, bad index) */
  RS_ETOOMANY_ERASURES = 2,  /* more erasures than parity blocks */
  RS_ENOMEM = 3,             /* host or device allocation failed */
  RS_ECUDA = 4,              /* a CUDA call failed */
  RS_ETIMEOUT = 5,           /* a device-side bounded wait gave up */
  RS_EUNSUPPORTED = 6        /* valid code outside the device path's limits */
} rs_status;

typedef enum {
  RS_READ_MIN = 0,  /* decode reads the first k surviving blocks (by index) */
  RS_READ_ALL = 1   /* decode reads every surviving block (§3.3, second remark) */
} rs_read_mode;

/* Library version (major * 10000 + minor * 100 + patch). */
int rs_version(void);

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next call on the same thread. */
const char *rs_last_error(void);

/* Create a code.  §3.1 (g(x)), §2.2 (Vandermonde), §2.3 (Cauchy).
 *   k >= 1, m in [1, 8] (m in [1, 4] for w = 16), k + m <= 64 and
 *   <= 2^w - 1, w in {8, 16},
 *   realization in rs_realization.
 * Builds the generator on the host and allocates a 4-byte device status
 * word on the current device.  *out receives the code (owned by the caller,
 * free with rs_destroy).  Errors: RS_EINVAL, RS_EUNSUPPORTED, RS_ENOMEM,
 * RS_ECUDA. */
rs_status rs_init(int k, int m, int w, int realization, rs_code **out);

/* Free a code (NULL is ignored).  Work still queued on a stream that uses
 * the code must have completed. */
void rs_destroy(rs_code *code);

/* RS_CAUCHY and RS_POLY_BITMATRIX only: packet size P in bytes (§2.3
 * projection; default 2048).
 * A block is a sequence of super-packets of w*P bytes; packet c of a
 * super-packet holds bit c of its 8P symbols.  P must be a positive
 * multiple of 128 (at most 1 MiB); block_bytes must then be a multiple of
 * w*P. */
rs_status rs_set_packet_bytes(rs_code *code, size_t packet_bytes);

/* Which survivors a decode reads (rs_read_mode, default RS_READ_MIN). */
rs_status rs_set_read_mode(rs_code *code, int mode);

/* Launch shape used by this code's kernels: consumer warps per CTA (1..16,
 * capped per kernel), shared-memory ring depth (2..64) and CTAs per SM
 * (1..4).  0 keeps the current value.  Set by the autotuner. */
rs_status rs_set_launch(rs_code *code, int consumer_warps, int depth, int ctas_per_sm);

/* Columns per thread of this code's kernels (not in the paper): 0 (the
 * default) picks the two-group kernels, 64 columns per thread, from blocks
 * of 256 KiB (symbol layout) or 8 KiB (packet layout) where they are
 * compiled; 1 always takes the one-group kernels (32 columns); 2 takes the
 * two-group kernels at every block size where they are compiled (else the
 * one-group ones).  Read when an encode or decode is prepared.  Set by the
 * autotuner.  Errors: RS_EINVAL. */
rs_status rs_set_groups(rs_code *code, int groups);

/* Encode one stripe: parity from data.  §3.2 Eq. 1 (polynomial: remainder of
 * x^m d(x) divided by g(x)), §2.1 (matrix: parity rows of G times d).
 *   data_ptrs: host array of k device pointers (read only);
 *   parity_ptrs: host array of m device pointers (written);
 *   block_bytes: bytes per block (any value >= 0; even for w = 16; a multiple
 *   of w*P for the packet realizations).  block_bytes = 0 is a no-op.
 * Errors: RS_EINVAL (null code/pointer, misalignment, size), RS_ECUDA. */
rs_status rs_encode(rs_code *code, const void *const *data_ptrs, void *const *parity_ptrs,
                    size_t block_bytes, void *stream);

/* Delta update of one stripe's parity after data block `index` changed.
 * §3.2's update remark: the code is linear, so the encode of the data
 * diff-blocks is the parity diff; with only block `index` changed by
 * delta = new XOR old, parity block j changes by P[j][index] * delta, where
 * P[:, index] is the encode of the unit data vector (x^(m+index) mod g(x)
 * for the polynomial code, the generator's parity column for the matrix
 * realizations).  Every realization and layout: delta and the parity
 * blocks are in the code's layout (packets for the bit-matrix
 * realizations).
 *   index: data block in [0, k);
 *   delta: device pointer to block_bytes bytes (read only);
 *   parity_ptrs: host array of m device pointers, updated in place
 *   (parity_j ^= P[j][index] * delta);
 *   block_bytes as for rs_encode.
 * Errors: RS_EINVAL (index, null, misalignment, overlap, size),
 * RS_EUNSUPPORTED, RS_ECUDA. */
rs_status rs_update(rs_code *code, int index, const void *delta, void *const *parity_ptrs, size_t block_bytes,
                    void *stream);

/* Decode one stripe: rebuild the erased blocks.  §3.3 (polynomial: Step 1
 * evaluates D(alpha^j) over the read survivors, Step 2 solves the small
 * Vandermonde system, inverted once per erasure pattern on the host), §2.1
 * (matrix realizations, solved here through the parity-check matrix).
 *   erasures: host array of n_erasures distinct block indices in [0, n);
 *   n_erasures in [0, m] (0 is a no-op, > m gives RS_ETOOMANY_ERASURES);
 *   block_ptrs: host array of n device pointers; survivors are read, erased
 *   blocks are written; block_bytes as for rs_encode.
 * Errors: RS_EINVAL, RS_ETOOMANY_ERASURES, RS_ECUDA. */
rs_status rs_decode(rs_code *code, const int *erasures, int n_erasures, void *const *block_ptrs,
                    size_t block_bytes, void *stream);

/* Bound of every device-side pipeline wait of this code's kernels, in
 * nanoseconds (0 = default, 2 s; at most 60 s).  A wait that runs out sets
 * the status word (see rs_poll_status) and the kernel returns early. */
rs_status rs_set_wait_limit(rs_code *code, unsigned long long nanoseconds);

/* Test hook for failure detection.  fault = 1: in the next launch of this
 * code, CTA 0's producer issues no copies, so that CTA's consumers run into
 * their bounded wait, record the timeout in the status word and return (no
 * copy is ever in flight for that CTA; other CTAs complete normally; the
 * affected tile's output is not written).  fault = 0 clears it.  Nothing
 * faults, traps or hangs: the context stays usable. */
rs_status rs_inject_fault(rs_code *code, int fault);

/* Read and clear the code's device status word (synchronises the device).
 * *device_status receives 0 or the kernel's error code; the return value is
 * RS_ETIMEOUT when the word was set, RS_OK otherwise. */
rs_status rs_poll_status(rs_code *code, int *device_status);

/* ------------------------------------------------------------------------
 * Batches: many stripe operations (any mix of codes, encodes and decodes of
 * any block sizes) in one persistent launch per kernel group.  Tiles of all
 * stripes are spread over one grid of (SMs x CTAs-per-SM) CTAs, so small
 * blocks do not pay one launch each.
 * ------------------------------------------------------------------------ */

typedef enum { RS_OP_ENCODE = 0, RS_OP_DECODE = 1 } rs_op_kind;

typedef struct {
  rs_code *code;       /* code of this stripe (must outlive the batch's launches) */
  int op;              /* rs_op_kind */
  int n_erasures;      /* RS_OP_DECODE: number of erased blocks (0..m) */
  int erasures[8];     /* RS_OP_DECODE: erased block indices in [0, n) */
  void *blocks[64];    /* n = k + m device pointers: data blocks then parity
                          blocks (same rules as rs_encode / rs_decode) */
  size_t block_bytes;  /* bytes per block of this stripe */
} rs_op;

/* Create a batch able to hold up to max_ops operations (1..2^20).
 * Allocates its device descriptor tables and a pinned staging buffer on
 * the current device (about 4.7 KB per op), and the side streams and
 * events that rs_batch_launch runs its kernel groups on.  Errors:
 * RS_EINVAL, RS_ENOMEM, RS_ECUDA. */
rs_status rs_batch_create(int max_ops, rs_batch **out);

/* Free a batch (NULL is ignored); its launches must have completed. */
void rs_batch_destroy(rs_batch *batch);

/* Launch shape for the batch's kernels (as rs_set_launch). */
rs_status rs_batch_set_launch(rs_batch *batch, int consumer_warps, int depth, int ctas_per_sm);

/* Columns per thread for the batch's ops (as rs_set_groups; the batch's
 * setting, not the codes', applies); read by rs_batch_set. */
rs_status rs_batch_set_groups(rs_batch *batch, int groups);

/* Validate and plan n_ops operations (§3.2 / §3.3 / §2.1 per op, as in
 * rs_encode / rs_decode), group them by kernel (at most 8 groups), and
 * upload the descriptor tables asynchronously on `stream`.  Host-side
 * errors name the failing op and leave the previous contents in place.
 * Launch on the same stream (or synchronise) so the upload is ordered
 * before the kernels.  The device tables are overwritten in place: a
 * launch of the previous contents must be on the same stream or complete
 * before this call's upload runs.  A CUDA graph that captured rs_batch_launch stays
 * valid after a later rs_batch_set as long as the new ops form the same
 * kernel groups in the same order (rs_batch_kernel_count and the op mix
 * unchanged): launch shapes are fixed and counts are read from device
 * memory. */
rs_status rs_batch_set(rs_batch *batch, const rs_op *ops, int n_ops, void *stream);

/* Enqueue the batch's kernels on `stream` (one persistent launch per
 * kernel group; no host synchronisation, no allocation).  The groups after
 * the first run on the batch's own side streams, forked from `stream` and
 * joined back into it: work queued on `stream` after this call waits for
 * every group, and the groups' kernels may overlap one another, as the ops
 * of one group already do -- so no op of a batch may read or write blocks
 * another op of the same batch writes. */
rs_status rs_batch_launch(rs_batch *batch, void *stream);

/* Number of kernel launches rs_batch_launch enqueues for the current set. */
int rs_batch_kernel_count(const rs_batch *batch);

/* Read and clear the batch's device status word (as rs_poll_status). */
rs_status rs_batch_poll_status(rs_batch *batch, int *device_status);

/* Batched block transfer.  The paper has no counterpart: moving the blocks
 * of a batch between host and device with one copy call per block costs a
 * host-side call per block, which limits a host thread feeding hundreds of
 * blocks per batch.  Copies range i, bytes[i] bytes from src[i] to dst[i],
 * for i < n, on `stream`: ranges of at least engine_min_bytes (0 = 4 MiB;
 * SIZE_MAX = none) as one copy-engine transfer each (no SMs used, but a
 * set-up cost per transfer), the smaller ones by one gather kernel launch
 * per 512 of them (no per-range cost, but it occupies SMs while the link
 * streams).  Every pointer is device memory or page-locked host
 * memory (cudaHostAlloc / cudaMallocHost / cudaHostRegister; on a system
 * with unified addressing it is mapped into the device address space and
 * read or written directly by the kernel at the host link's bandwidth);
 * pageable memory is rejected.
 * Pointers 16-byte aligned; any byte count; each range lies inside one
 * allocation (as for cudaMemcpy).  Ranges must not overlap one another's
 * destinations.  The caller keeps the memory alive and unchanged
 * until the stream reaches the copy.  No device memory is allocated (the
 * kernel's descriptors travel as kernel parameters), so the call can be
 * captured in a CUDA graph.  Errors: RS_EINVAL (null, misaligned, overlapping within a
 * range, pageable or unknown memory), RS_ENOMEM, RS_ECUDA. */
rs_status rs_copy_blocks(void *const *dst, const void *const *src, const size_t *bytes, int n,
                         size_t engine_min_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free batched encode.  The paper has no counterpart.  Some
 * callers cannot allocate device memory at the moment they encode:
 * allocator and memory-pool callbacks (a caching allocator that encodes the
 * blocks it evicts) must not re-enter the allocator they belong to;
 * embedders that reserve the whole device memory budget at start-up forbid
 * allocations afterwards; latency-critical paths cannot afford cudaMalloc /
 * cudaFree, which may synchronise the device.  rs_init and rs_batch_create
 * allocate (status word, descriptor tables); this call allocates nothing:
 * all scratch the batched kernel needs (descriptor tables, pointer table,
 * a status word) lives in one fixed 256 KiB static device array, reserved on
 * every GPU that loads the library until the process exits, and the tables
 * reach it through small upload kernels that carry them as kernel
 * parameters.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  The caller passes only the blocks.
 *
 * Encodes n_stripes stripes of the polynomial RS(k, m) code over GF(2^w)
 * (§3.2 Eq. 1 per stripe) with one persistent encode launch on `stream`:
 *   data_ptrs:   n_stripes * k device pointers, stripe-major (stripe s uses
 *                data_ptrs[s*k .. s*k+k-1]);
 *   parity_ptrs: n_stripes * m device pointers, stripe-major;
 *   block_bytes: n_stripes block sizes (0 skips the stripe);
 *   device_status: NULL, or a 4-byte aligned device pointer to an int the
 *                caller has set to 0: a device-side wait that gives up (the
 *                2 s bound of the staging pipeline) stores a nonzero code
 *                there and the affected tiles' parity is not written.  With
 *                NULL the code goes to the array's own status word, which no
 *                call reports.
 * Block rules as for rs_encode; the bytes written equal rs_encode's for the
 * same stripes.  Limits: those of rs_init, and the tables must fit the
 * array: 256 + (S * 56 rounded up to 256) + S * (k + m) * 8 bytes <= 262144
 * for S non-empty stripes (e.g. up to 1500 stripes of RS(10,4)); larger
 * requests return RS_EINVAL with the sizes in rs_last_error.
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current), and the first call for
 * each (w, m) on a device sets its encode kernel's shared-memory size
 * attribute; later calls skip both steps.  Make those first calls before
 * any stream capture begins.  The array
 * is shared by all calls on a device and keeps the last call's contents:
 * each call clears the status word and rewrites the tables before its
 * kernel runs, so calls whose work overlaps on the GPU race -- order them
 * on one stream or synchronise between them.
 * Errors: RS_EINVAL, RS_EUNSUPPORTED, RS_ECUDA. */
rs_status rs_poly_encode_stripes_noalloc(int k, int m, int w, int n_stripes, const void *const *data_ptrs,
                                         void *const *parity_ptrs, const size_t *block_bytes,
                                         int *device_status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RS_GB300_H */
