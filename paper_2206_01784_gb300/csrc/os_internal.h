// Host-side interface between the C ABI (os_api.cu) and the kernel
// translation units. Plain structs of device pointers and sizes.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace onesweep {

// Phase 1 + 2 (Section 3, "Upfront histogram kernel", "Exclusive sum kernel").
struct HistArgs {
  const void* keys;          // n keys (device)
  uint64_t n;
  int flip;                  // float keys: apply the sign-flip before taking digits
  int num_places;            // p
  int radix_bits;            // d: place i covers bits [begin_bit + d*i, min(+d, end_bit)); 5..8
  int begin_bit;
  int end_bit;
  uint32_t* hist;            // [p][256] zeroed by the caller (device); 2^d bins used per row
  uint32_t* offsets;         // [p][256] written by the last block (device)
  uint32_t* done_counter;    // zeroed by the caller (device)
  uint32_t* clear;           // words to zero on the way (status slab of pass 0), may be null
  uint64_t clear_words;
  uint32_t* skew;            // [p] set to 1 where one digit holds over 1/16 of the keys (may be null)
  uint32_t top_xor;          // signed keys: high bit of the top place's digit inverted (else 0)
  uint32_t descending;       // offsets (and the reported histograms) for complemented digits
};

// Phase 3, one digit-binning pass (Section 3, "Chained scan digit-binning kernel").
struct PassArgs {
  const void* keys_in;
  void* keys_out;
  const uint32_t* vals_in;   // null for keys only
  uint32_t* vals_out;
  uint32_t n;
  uint32_t num_tiles;
  int shift;                 // digit = (ordered key >> shift) & mask
  uint32_t mask;
  int flip_in;               // apply the float sign-flip to loaded keys
  int flip_out;              // undo it on stored keys
  int use_bulk;              // inputs 16-byte aligned: stage full tiles with bulk copies
  const uint32_t* bin_offsets;  // [256] global bin offsets of this place
  uint32_t* status;          // [num_tiles][256] status counters, zeroed
  uint32_t* status_clear;    // slab of the next launch, to zero (may be null) ...
  uint32_t status_clear_rows;  // ... rows 0 .. status_clear_rows-1 of it (>= num_tiles)
  uint32_t* tile_counter;    // zeroed; hands out tile ids in launch order
  uint32_t* error;           // device status word
  uint32_t spin_limit;       // look-back polls before giving up
  int64_t fault_tile;        // test hook: tile that never publishes (-1 = none)

  // Strips (Section 3, "Handling very large problems"): a pass over more than
  // one strip is one launch per strip. keys_in / vals_in point at the strip,
  // n is the strip's length and bin_offsets hold the strip's bin bases (where
  // its first key of each digit lands); out_total is the whole array's length
  // (the output bound). The strip's last tile writes the next strip's bases to
  // carry_out (null when there is no next strip).
  uint32_t out_total;
  uint32_t* carry_out;

  // Segmented mode (os_sort_batch); seg_offsets == nullptr means one array of
  // n keys. Each segment is its own sort: its tiles form one look-back chain
  // and it has its own bin offsets.
  const uint64_t* seg_offsets;   // [S+1] segment boundaries (device)
  const uint32_t* tile_base;     // [S+1] first tile of each segment's chain
  const uint32_t* tile_seg;      // [tiles] segment of each tile
  const uint32_t* total_tiles;   // device word: tiles in this pass
  uint32_t offsets_stride;       // words between two segments' bin offsets

  // Skewed-place flags from the histogram pass (null: none); the flag of
  // segment s (0 for one array) is skew_flags[s * skew_stride].
  const uint32_t* skew_flags;
  uint32_t skew_stride;
  uint32_t digit_xor;            // signed keys, top place: invert the digit's high bit (else 0)
};

// Segmented sort: the plan, per-segment histograms and the one-block sort of
// small segments (os_batch.cu).
struct BatchArgs {
  const void* keys_in;
  void* keys_out;
  const uint32_t* vals_in;
  uint32_t* vals_out;
  const uint64_t* seg_offsets;   // [S+1]
  uint32_t num_segments;
  uint64_t n_total;
  int flip;                      // float keys
  int num_places;
  int begin_bit;
  int end_bit;
  uint32_t small_max;            // segments up to this length are sorted in one block
  uint32_t tile_keys;            // binning tile of the large segments
  uint32_t hist_chunk;           // keys per histogram work item
  uint32_t max_tiles;            // capacity of tile_seg
  uint32_t max_items;            // capacity of hist_seg
  uint32_t* tile_base;           // [S+1]
  uint32_t* tile_seg;            // [max_tiles]
  uint32_t* hist_base;           // [S+1]
  uint32_t* hist_seg;            // [max_items]
  uint32_t* totals;              // [0] binning tiles, [1] histogram items
  uint32_t* seg_done;            // [S] zeroed
  uint32_t* seg_hist;            // [S][p][256] zeroed
  uint32_t* seg_bin_offsets;     // [S][p][256]
  uint32_t* seg_skew;            // [S][p] skewed-place flags
  uint32_t top_xor;              // signed keys: high bit of the top place's digit inverted (else 0)
  uint32_t descending;           // bin by the complemented digit of every place
  uint32_t* error;
  uint32_t* clear;               // status slab of the first pass, to zero
  uint64_t clear_words;
};

constexpr uint32_t kErrBadSegments = 2u;  // device status word bit: invalid segment offsets

cudaError_t launch_batch_plan(const BatchArgs& b, cudaStream_t s);
cudaError_t launch_batch_histogram(int key_bits, const BatchArgs& b, cudaStream_t s);
cudaError_t launch_batch_local_sort(int key_bits, bool pairs, const BatchArgs& b, cudaStream_t s);
uint32_t batch_local_capacity(int key_bits, bool pairs);

// Active binning variant for a key width / payload / size bucket, and the
// tile size of a variant.
int binning_config(int key_bits, bool pairs, int bucket);
uint32_t tile_keys_for(int key_bits, bool pairs, int cfg);

int sort_on_workspace(int key_type, const void* keys_in, void* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                      uint64_t n, int begin_bit, int end_bit, void* ws, size_t ws_bytes, void* stream);

cudaError_t launch_histogram(int key_bits, const HistArgs& a, int num_sms, cudaStream_t s);
// Launches variant cfg of the binning kernel (the variant a plan was made with).
cudaError_t launch_binning(int key_bits, bool pairs, int cfg, const PassArgs& a, cudaStream_t s,
                           int radix_bits = 8);

}  // namespace onesweep
