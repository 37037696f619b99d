/*
 * onesweep.h - C ABI of the GB300 Onesweep LSD radix sort.
 *
 * Implements the sort of Adinets and Merrill, "Onesweep: A Faster Least
 * Significant Digit Radix Sort for GPUs" (arXiv 2206.01784):
 *   phase 1  one pass computes the digit histograms of every digit place
 *            (Section 3, "Upfront histogram kernel"; Figure 5);
 *   phase 2  an exclusive prefix sum of each histogram gives the global bin
 *            offsets (Section 3, "Exclusive sum kernel");
 *   phase 3  p single-pass chained-scan digit-binning passes, least
 *            significant place first (Section 3, "Chained scan digit-binning
 *            kernel"; Figures 6-8).
 * The problem solved is the paper's: an ascending, stable sort of keys held in
 * GPU global memory, optionally carrying 32-bit payload values (Section 1;
 * Section 4 evaluates 32/64-bit keys and 32-bit values).
 *
 * Conventions shared by every call:
 *  - Pointers named *_in / *_out / ws are DEVICE pointers; the caller owns all
 *    of them. The library never allocates device memory: scratch space is the
 *    caller's workspace `ws` of at least os_sort_workspace_bytes() bytes.
 *  - Keys are raw bit patterns: uint32 (OS_KEY_U32), uint64 (OS_KEY_U64),
 *    IEEE-754 binary32 (OS_KEY_F32) or binary64 (OS_KEY_F64), two's-complement
 *    int32 (OS_KEY_I32) or int64 (OS_KEY_I64). Signed keys are ordered as
 *    their bits with the sign bit inverted (Section 3's "magnitude-preserving
 *    conversion" for signed types); float keys are
 *    ordered through the bijective sign-flip (negative keys: all bits
 *    inverted; others: sign bit set), so -0.0 sorts before +0.0 and NaNs sort
 *    by bit pattern (negative NaNs first, positive NaNs last). Output keys
 *    carry the input bits unchanged.
 *  - [begin_bit, end_bit) selects the key bits sorted on (of the sign-flipped
 *    bits for float and signed keys), 0 <= begin_bit <= end_bit <= key width. Digit
 *    places are 8 bits wide, start at begin_bit and go upward; the last place
 *    is narrower when the range is not a multiple of 8. begin_bit == end_bit
 *    copies the input.
 *  - Sorting is stable: equal keys keep their input order, and values follow
 *    their keys.
 *  - n must be below 2^32 (output positions are 32-bit); larger n returns
 *    OS_ERR_TOO_LARGE. The chained scan keeps 30-bit counts, so passes over
 *    2^30 keys or more run strip by strip (Section 3, "Handling very large
 *    problems"; onesweep_debug.h can shorten strips for tests).
 *  - Inputs are never modified. Input, output and workspace ranges must not
 *    overlap (OS_ERR_INVALID_ARG). Key pointers must be aligned to the key
 *    width and value pointers to 4 bytes.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls only
 *    enqueue work and return after host-side validation; results are ready
 *    when the stream reaches them. Errors found on the device (a look-back
 *    wait that ran past its limit) are reported by os_workspace_status().
 *  - Calls that share a workspace must not overlap on the GPU.
 */
#ifndef ONESWEEP_H
#define ONESWEEP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OS_API __attribute__((visibility("default")))
#else
#define OS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OS_KEY_U32 = 0,
    OS_KEY_U64 = 1,
    OS_KEY_F32 = 2,
    OS_KEY_F64 = 3,
    OS_KEY_I32 = 4,
    OS_KEY_I64 = 5
} os_key_type;

/*
 * OR'd into any key_type argument: stable descending order - keys from the
 * largest sorted-on field down, equal keys still in their input order. The
 * paper sorts ascending only (Section 4); each digit place here bins by the
 * complement of its digit within the place, which costs nothing (the same
 * XOR that orders signed keys). For float keys, +0.0 comes before -0.0 and
 * NaNs follow their bit patterns, reversed.
 */
#define OS_SORT_DESCENDING 0x100

typedef enum {
    OS_OK = 0,
    OS_ERR_INVALID_ARG = 1, /* bad key type, bit range, pointer, alignment or overlap */
    OS_ERR_TOO_LARGE = 2,   /* n >= 2^32 */
    OS_ERR_WORKSPACE = 3,   /* workspace missing or smaller than required */
    OS_ERR_CUDA = 4,        /* a CUDA call or kernel launch failed */
    OS_ERR_TIMEOUT = 5,     /* a chained-scan look-back wait ran past its limit */
    OS_ERR_SCRATCH_LIMIT = 6 /* os_sort_noalloc: the sort needs more than its fixed scratch */
} os_status;

/* Where the parts of a sort's workspace sit (byte offsets from ws). */
typedef struct {
    size_t total_bytes;        /* what os_sort_workspace_bytes() returns */
    size_t status_offset[2];   /* the two status-counter slabs (pass i uses slab i % 2) */
    size_t histogram_offset;   /* uint32 [places][256] digit counts */
    size_t bin_offset_offset;  /* uint32 [places][256] global bin offsets */
    size_t alt_keys_offset;    /* ping-pong key buffer */
    size_t alt_values_offset;  /* ping-pong value buffer (0 bytes for keys only) */
    uint32_t tile_keys;        /* keys per binning tile */
    uint32_t num_tiles;        /* tiles per binning pass */
    uint32_t num_places;       /* p */
} os_workspace_layout;

/*
 * Workspace bytes for sorting n keys of key_type over [begin_bit, end_bit)
 * with value_bytes = 0 (keys only) or 4 (uint32 values). Returns 0 for
 * invalid arguments. The workspace holds the digit histograms and bin offsets
 * (Section 3, phases 1-2), two slabs of 32-bit status counters, one per
 * (tile, digit) (Section 3, Figure 6), and the ping-pong key/value buffers.
 */
OS_API size_t os_sort_workspace_bytes(int key_type, uint64_t n, int value_bytes, int begin_bit, int end_bit);

/* Fills *layout for the same arguments. Returns OS_OK or OS_ERR_INVALID_ARG. */
OS_API int os_sort_workspace_layout(int key_type, uint64_t n, int value_bytes, int begin_bit, int end_bit,
                             os_workspace_layout *layout);

/*
 * Sorts n keys (Section 3, all three phases). keys_in: n keys (device);
 * keys_out: n keys (device), receives the stable ascending order. Returns an
 * os_status.
 */
OS_API int os_sort_keys(int key_type, const void *keys_in, void *keys_out, uint64_t n, int begin_bit, int end_bit,
                 void *ws, size_t ws_bytes, void *stream);

/*
 * Sorts n (key, uint32 value) pairs by key (Section 3; Section 4 sorts
 * 32-bit keys with 32-bit values). vals_in / vals_out: n uint32 (device);
 * each value moves with its key. Returns an os_status.
 */
OS_API int os_sort_pairs(int key_type, const void *keys_in, void *keys_out, const uint32_t *vals_in, uint32_t *vals_out,
                  uint64_t n, int begin_bit, int end_bit, void *ws, size_t ws_bytes, void *stream);

/*
 * The same sorts for arrays held in HOST memory. keys_in / vals_in: n keys
 * (uint32 values) in host memory, read; keys_out / vals_out: n keys (values)
 * in host memory, written with the stable ascending order. The call enqueues
 * on `stream`, in order, the uploads into staging buffers inside ws, the
 * sort (os_sort_keys / os_sort_pairs on those buffers) and the downloads; the
 * output is complete when the stream gets past the call (cudaStreamSynchronize,
 * or os_workspace_status(ws, stream)). Host buffers should be page-locked
 * (cudaHostAlloc / cudaHostRegister) for the copies to run asynchronously;
 * pageable buffers work, but the call then waits for its copies. ws:
 * os_sort_host_workspace_bytes() bytes of DEVICE memory (16-byte aligned);
 * it begins with the sort's own workspace, so os_workspace_status(ws, ...)
 * reports device-side errors as for os_sort_keys. Host ranges must not
 * overlap (OS_ERR_INVALID_ARG). Not part of the paper: the sort as a caller
 * with data in host memory uses it (two calls on two streams with two
 * workspaces overlap one array's copies with another's sort).
 */
OS_API size_t os_sort_host_workspace_bytes(int key_type, uint64_t n, int value_bytes, int begin_bit, int end_bit);
OS_API int os_sort_keys_host(int key_type, const void *keys_in, void *keys_out, uint64_t n, int begin_bit,
                             int end_bit, void *ws, size_t ws_bytes, void *stream);
OS_API int os_sort_pairs_host(int key_type, const void *keys_in, void *keys_out, const uint32_t *vals_in,
                              uint32_t *vals_out, uint64_t n, int begin_bit, int end_bit, void *ws, size_t ws_bytes,
                              void *stream);

/*
 * How the host-memory sorts above move data between host and device memory
 * (process-wide; not part of the paper). OS_HOST_COPY_ENGINES (the default):
 * cudaMemcpyAsync on the call's stream. OS_HOST_COPY_LINK: copy kernels on the
 * call's stream that read or write the host buffers directly through their
 * device mapping - host ranges that are page-locked and mapped from their
 * first to their last byte (cudaHostAlloc, or cudaHostRegister with
 * cudaHostRegisterMapped) and start 16-byte aligned (the last bytes of
 * a count that is not a multiple of 16 still go through the copy engines);
 * any other buffer takes the copy engines. Results are the same in both
 * modes. os_set_host_copy_mode returns OS_OK, or OS_ERR_INVALID_ARG for an
 * unknown mode; os_get_host_copy_mode returns the mode in force.
 */
#define OS_HOST_COPY_ENGINES 0
#define OS_HOST_COPY_LINK 1
OS_API int os_set_host_copy_mode(int mode);
OS_API int os_get_host_copy_mode(void);

/*
 * Segmented (batched) sort: num_segments independent arrays held back to
 * back, segment s = [seg_offsets[s], seg_offsets[s+1]), each sorted on its
 * own, in one call of a few launches whatever the number of segments (each
 * segment gets its own Section 3 histograms, bin offsets and look-back
 * chain; segments of up to one block's capacity are sorted in shared
 * memory). seg_offsets: num_segments + 1 uint64 (DEVICE), nondecreasing,
 * seg_offsets[num_segments] <= n_total, each segment shorter than 2^30 keys;
 * keys outside every segment are not written. n_total < 2^31. The offsets
 * are read on the device only, so a call can be captured in a CUDA graph;
 * invalid offsets are reported by os_workspace_status() as
 * OS_ERR_INVALID_ARG (nothing is sorted). vals_in / vals_out: NULL for keys
 * only, else n_total uint32 each. ws: os_sort_batch_workspace_bytes() bytes.
 * Not part of the paper: the batching the paper's single sort is built into.
 */
OS_API size_t os_sort_batch_workspace_bytes(int key_type, uint64_t n_total, int num_segments, int value_bytes,
                                            int begin_bit, int end_bit);
OS_API int os_sort_batch(int key_type, const void *keys_in, void *keys_out, const uint32_t *vals_in,
                         uint32_t *vals_out, const uint64_t *seg_offsets, int num_segments, uint64_t n_total,
                         int begin_bit, int end_bit, void *ws, size_t ws_bytes, void *stream);

/*
 * Phases 1 and 2 only (Section 3, "Upfront histogram kernel" and
 * "Exclusive sum kernel"): the digit counts of every place of the n keys and
 * their exclusive prefix sums. hist_out and offsets_out are device arrays of
 * uint32 [p][256] (either may be NULL). ws: a workspace sized by
 * os_sort_workspace_bytes(key_type, n, 0, begin_bit, end_bit).
 */
OS_API int os_digit_histograms(int key_type, const void *keys_in, uint64_t n, int begin_bit, int end_bit,
                        uint32_t *hist_out, uint32_t *offsets_out, void *ws, size_t ws_bytes, void *stream);

/*
 * Waits for `stream`, then reports what the device recorded in the
 * workspace's status word during the last call that used it: OS_OK,
 * OS_ERR_TIMEOUT (a look-back wait gave up; the output is not valid) or
 * OS_ERR_CUDA (the stream reported an error).
 */
OS_API int os_workspace_status(const void *ws, void *stream);

/* A static, human-readable name for an os_status value. */
OS_API const char *os_status_string(int status);

/*
 * What this library was built for (not part of the method). os_build_info()
 * returns a static string naming the virtual architectures its device code
 * was compiled for ("cuda_arch_list=1030" for sm_103a); it needs no GPU.
 * os_binary_version() asks the driver for the architecture of the device code
 * it loaded on the current device (cudaFuncAttributes::binaryVersion, 103 for
 * sm_103a), or returns a negative CUDA error code.
 */
OS_API const char *os_build_info(void);
OS_API int os_binary_version(void);

/*
 * os_sort_noalloc - the same sort as os_sort_keys / os_sort_pairs for callers
 * that cannot allocate device memory. The paper has no counterpart; this is a
 * convenience of this library.
 *
 * Who needs it: code that runs where every byte of device memory already
 * belongs to someone else's allocator (a host framework's memory pool with a
 * hard budget, a plugin that must not allocate behind its host's back), or
 * where a cudaMalloc/cudaFree would implicitly synchronize the device and
 * stall a latency-critical pipeline. Such callers can pass their keys and
 * values but cannot hand the sort a workspace.
 *
 * The scratch the sort needs (digit histograms, status counters, ping-pong
 * buffers) lives in one fixed 16 MiB array of static device memory inside
 * this library, so this call allocates nothing. Every GPU that loads the
 * library holds those 16 MiB until the process exits. That bounds the
 * problem size: a call whose workspace (os_sort_workspace_bytes) would exceed
 * 16 MiB returns OS_ERR_SCRATCH_LIMIT and does nothing. Up to 2^20 keys always
 * fit, for every key type, with or without values.
 *
 * Arguments as os_sort_pairs; vals_in and vals_out both NULL sorts keys only
 * (exactly one of them NULL is OS_ERR_INVALID_ARG). The sort runs on the
 * current device and `stream` must belong to it. The first call on a device -
 * and the first after that device's context was recreated, e.g. by
 * cudaDeviceReset - looks up the device's copy of the scratch array
 * (cudaGetSymbolAddress), so make that first call before any stream capture
 * begins. All calls share the one array per device and each call leaves its
 * contents behind (the sort re-initialises what it needs): calls that may
 * overlap on the GPU (different streams without ordering between them) race
 * on it and must be serialized by the caller. Device-side errors are reported
 * by os_workspace_status() given the scratch address returned through
 * `scratch_out` (may be NULL).
 */
OS_API int os_sort_noalloc(int key_type, const void *keys_in, void *keys_out, const uint32_t *vals_in,
                           uint32_t *vals_out, uint64_t n, int begin_bit, int end_bit, void *stream,
                           const void **scratch_out);

/*
 * Tile geometry of the digit-binning kernel (tuning, not part of the method).
 * There are os_num_tile_configs() geometries per key width and payload
 * (keys only: value_bytes 0, pairs: 4); os_tile_config_keys() gives the keys
 * per tile of one (0 for invalid arguments). os_set_tile_config() selects the
 * geometry later calls use (process-wide, applied at launch time); results
 * are identical under every geometry. Workspaces are sized for the smallest
 * tile, so a workspace sized once fits every geometry. os_set_tile_config
 * returns OS_OK or OS_ERR_INVALID_ARG; os_get_tile_config returns the active
 * geometry or -1.
 */
OS_API int os_num_tile_configs(void);
OS_API int os_tile_config_keys(int key_bits, int value_bytes, int cfg);
OS_API int os_set_tile_config(int key_bits, int value_bytes, int cfg);
OS_API int os_get_tile_config(int key_bits, int value_bytes);

/*
 * The active geometry is kept per size bucket too (os_num_size_buckets()
 * buckets; os_size_bucket(n) names the bucket of a sort of n keys, and a
 * batch uses the bucket of its mean segment length). os_set_tile_config sets
 * every bucket; these set or read one (os_get_tile_config reads the largest).
 * Same return conventions as above.
 */
OS_API int os_num_size_buckets(void);
OS_API int os_size_bucket(uint64_t n);
OS_API int os_set_tile_config_bucket(int key_bits, int value_bytes, int bucket, int cfg);
OS_API int os_get_tile_config_bucket(int key_bits, int value_bytes, int bucket);

/*
 * The process-wide digit width d (bits per digit place; Section 3, and the
 * d sweep of Section 4, Table 2) per size bucket, used by single-array sorts
 * whose per-call options leave radix_bits at 0 (no options, or
 * os_sort_options.radix_bits == 0); 8 until set. A sort that names a tile
 * variant other than 4 and leaves radix_bits at 0 uses 8; batches always use
 * 8. radix_bits: 5-8, else OS_ERR_INVALID_ARG. The get call returns the
 * width, or -1 for invalid arguments. The sorted output never depends on d.
 */
OS_API int os_set_radix_bits_bucket(int key_bits, int value_bytes, int bucket, int radix_bits);
OS_API int os_get_radix_bits_bucket(int key_bits, int value_bytes, int bucket);

/*
 * Launch timing for benchmarks (not part of the method). os_profile_start
 * makes every later kernel launch of the library record a CUDA event pair on
 * its own stream, for up to `capacity` launches. os_profile_stop waits for
 * those events, writes up to `max` records to `out` (host array), stores how
 * many launches were recorded in *count, releases the events and switches
 * recording off. Process-wide (the recording table is guarded by a lock, but
 * the timings mean something only for launches from one thread). Both return
 * an os_status.
 */
typedef struct {
    int kernel;   /* 0 = histogram (phases 1-2), 1 = digit binning (phase 3),
                     2 = batch plan, 3 = batch one-block sort of small segments */
    int pass;     /* digit place of a binning launch, -1 for the histogram */
    float ms;     /* device time between the pair of events */
} os_launch_time;

OS_API int os_profile_start(int capacity);
OS_API int os_profile_stop(os_launch_time *out, int max, int *count);

/*
 * Per-call options (not part of the method): the same sorts as os_sort_keys,
 * os_sort_pairs and os_sort_batch with the binning variant chosen by the
 * caller rather than read from the process-wide table above, so that
 * concurrent callers (several host threads, several streams) can each use
 * their own. opt == NULL or opt->tile_config == -1 means the process-wide
 * choice for the sort's size bucket; any other value must be below
 * os_num_tile_configs() (else OS_ERR_INVALID_ARG). Results are identical for
 * every variant. The library holds no other per-call state: calls on
 * different streams with different workspaces may run concurrently from any
 * number of host threads.
 *
 * radix_bits: bits per digit place d (Section 3; Section 4, Table 2 measures
 * d = 5..9). 0 means the process-wide choice (os_set_radix_bits_bucket; 8,
 * with 256 bins and p = ceil(bits / 8) passes, until set); 5, 6 or 7 sort
 * with 2^d bins in ceil(bits / d) passes, using tile variant
 * 4 (tile_config must then be -1 or 4) and single arrays only
 * (os_sort_batch_ex rejects them). Any other value: OS_ERR_INVALID_ARG. The
 * sorted output is the same for every d; only the number and cost of the
 * passes change. Workspace sizes do not depend on d.
 */
typedef struct {
    int tile_config;
    uint32_t radix_bits;
} os_sort_options;

OS_API int os_sort_keys_ex(int key_type, const void *keys_in, void *keys_out, uint64_t n, int begin_bit,
                           int end_bit, void *ws, size_t ws_bytes, void *stream, const os_sort_options *opt);
OS_API int os_sort_pairs_ex(int key_type, const void *keys_in, void *keys_out, const uint32_t *vals_in,
                            uint32_t *vals_out, uint64_t n, int begin_bit, int end_bit, void *ws, size_t ws_bytes,
                            void *stream, const os_sort_options *opt);
OS_API int os_sort_batch_ex(int key_type, const void *keys_in, void *keys_out, const uint32_t *vals_in,
                            uint32_t *vals_out, const uint64_t *seg_offsets, int num_segments, uint64_t n_total,
                            int begin_bit, int end_bit, void *ws, size_t ws_bytes, void *stream,
                            const os_sort_options *opt);

#ifdef __cplusplus
}
#endif

#endif /* ONESWEEP_H */
