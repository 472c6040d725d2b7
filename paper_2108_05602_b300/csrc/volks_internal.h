// Internal declarations shared by the host driver (volks_api.cu,
// volks_plan.cu, volks_noalloc.cu) and the kernels (volks_kernels.cu).
// Not part of the ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vk {

constexpr int kTile = 32;          // APs per search tile (largest window)
constexpr int kMaxWinLog = 5;      // windows 1, 2, 4, 8, 16, 32
constexpr int kMaxSegPerTile = 63; // 32 + 16 + 8 + 4 + 2 + 1
constexpr int kMaxDesc = 64;       // ranges per launch (kernel parameter block)

// Window-matched group found on the device (a9), before the host's
// cross-baseline step.
struct DevCand {
  int32_t bl, dm_idx, win_log, seg;
  int32_t g0, g1, n_windows;
  uint32_t lin;                    // q * M + m of the representative's peak
  float P;
  float _pad;
  double rho, z;
};

// One work range: one segment restricted to a contiguous chunk of its DM
// trials.  Passed to the kernels inside a __grid_constant__ parameter block.
struct SegDesc {
  const float2* xn;                // [n_bl][n_f][n_ap] normalised, calibrated
  const int32_t* shifts;           // [n_dm][n_f] of this chunk
  const int32_t* nvalid;           // [n_dm] of this chunk
  const float2* tw_n;              // W_{n_f}^i, i < n_f
  const float2* tw_m;              // W_M^i, i < M
  unsigned long long* keys;        // [n_bl][n_dm][seg_per_bd] of this chunk
  double* stats;                   // [n_bl][n_dm_total][n_win][2] (all DMs of the segment)
  uint32_t* bits;                  // [n_bl][n_dm][word_per_bd] of this chunk
  DevCand* cand;                   // window-matched groups of the segment
  unsigned int* count;
  unsigned int cap;
  int seg_id;
  long long seg_per_bd, word_per_bd;
  long long base;                  // first work unit of this range within its launch
  int n_bl, n_ap, n_f, n_dm, n_dm_total, d0, pad_delay, M, n_tiles;
  int n_win, n_eff, min_windows, win_mask;
  int win_log[kMaxWinLog + 1];     // by window index
  int win_off[kMaxWinLog + 1];     // segment offset, by window index
  int word_off[kMaxWinLog + 1];    // bit-word offset, by window index
  int win_off_l[kMaxWinLog + 1];   // segment offset, by log2(window)
  double thresh;
};

// Segments of window 2^l in a series of nv dedispersed APs, and the first
// AP of segment s: back to back (stride 2^l) or sliding (stride 1).
__host__ __device__ inline int seg_count(int nv, int l, int slide) {
  nv = nv > 0 ? nv : 0;
  return slide ? (nv >= (1 << l) ? nv - (1 << l) + 1 : 0) : nv >> l;
}
__host__ __device__ inline int seg_start(int s, int l, int slide) { return slide ? s : s << l; }

// SegDesc.win_mask: bits 0-5 the searched windows (bit l: 2^l APs); for
// sliding segments bit 16 is set and bits 8-15 hold the number of AP phases
// of the search units (the largest window).  Every window test reads the
// low bits only.
constexpr int kWinBits = 0x3f;
constexpr int kSlideBit = 1 << 16;
__host__ __device__ inline int desc_slide(int win_mask) { return (win_mask >> 16) & 1; }
__host__ __device__ inline int desc_phases(int win_mask) {
  const int n = (win_mask >> 8) & 0xff;
  return n > 0 ? n : 1;
}

// A launch over up to kMaxDesc ranges.  counter == nullptr: unit
// blockIdx.x + unit0 per CTA (per thread for the match kernel); otherwise
// the search kernel is persistent and pulls units from *counter (zeroed
// before the launch) until `total`.
struct Batch {
  unsigned long long* counter;
  unsigned int* err;               // tensor-core kernel: set non-zero if a bounded wait gave up
  long long total;
  long long unit0;
  int n_desc;
  SegDesc d[kMaxDesc];
};

// Work split of the search kernel: 32 * n1 threads, fold band folds.
struct SearchVariant {
  int n1, fold;
};

struct PrepArgs {
  const float2* vis;               // [n_pol][n_bl][n_ap][n_f]
  const float* autos;              // [n_pol][n_st][n_ap][n_f] auto-spectrum power, or NULL
  const int2* bl_st;               // [n_bl] station pair of each baseline (with autos)
  float2* xn;                      // [n_bl][n_f][n_ap]  (normalised, calibrated, polarisations summed)
  double* part;                    // [n_rows][n_tchunk][n_f] partial sums of |S|^2 (rows = (pol, bl))
                                   // or of a^2 (rows = (pol, station)) with autos
  const double2* phasor;           // [n_pol][n_bl][n_f] calibration phasor (FP64)
  float2* gain;                    // [n_pol][n_bl][n_f]
  int n_bl, n_ap, n_f, n_chan, n_tchunk, tchunk;
  int n_pol, n_st;
  int normalize, skip_first_chan;
};

// Single-range search arguments (one CTA per work unit, no counter).
struct SearchArgs {
  const float2* xn;
  const int32_t* shifts;
  const int32_t* nvalid;
  const float2* tw_n;
  const float2* tw_m;
  unsigned long long* keys;
  int n_bl, n_ap, n_f, n_dm, pad_delay, M;
  int win_mask;
  int win_off[kMaxWinLog + 1];     // by log2(window)
  long long seg_per_bd;
  int n_tiles;
  int fold;
};

// Set the calling thread's message returned by volks_last_error().
void set_last_error(const char* msg);

// Arithmetic of the rate search that a (n_f, pad_rate, precision) search
// actually runs: the tensor-core kernels cover 2-D searches (pad_rate 4)
// of bands with a tensor-core work split (n_f >= 256); everything else
// runs the FP32 kernel (VOLKS_FP32).
int effective_precision(int n_f, int pad_rate, int precision);
// Default work split for a band of n_f points at an effective precision
// (fold_override > 0 forces that fold where a variant with it exists).
SearchVariant default_variant(int n_f, int precision, int fold_override);
// The variants compiled for a band of n_f points at an effective precision
// (at most 4).
int search_variants(int n_f, int precision, SearchVariant* out);
// Search units (CTAs) of one range.
long long search_units(const SegDesc& d, SearchVariant v);
// CTAs per SM of the search kernel for this variant (0 on error).
int search_occupancy(SearchVariant v, int pad_rate, int precision);
// True when a tensor-core search kernel is compiled for this split.
bool mma_supported(SearchVariant v, int pad_rate, int precision);

// Launchers (return the launch's cudaError_t).
cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s, int* n_launch);
// Persistent (b.counter != nullptr; grid_ctas CTAs) or one CTA per unit;
// all ranges of b share n_f, pad_rate and the variant; b.total = units.
// precision: the effective precision; reduced precisions run the
// persistent tensor-core kernel (b.counter and b.err required).
cudaError_t launch_search_batch(Batch& b, SearchVariant v, int pad_rate, int precision, int grid_ctas,
                                cudaStream_t s, int* n_launch);
cudaError_t launch_search_mma(Batch& b, SearchVariant v, int precision, int grid_ctas, cudaStream_t s,
                              int* n_launch);
// Checking aid: one 128-delay-cell block of the rate GEMM of window 2^l
// (y: device complex64 [32][128], tw_m: W_M^i, i < M) -> out: device
// float [128][256], the job's accumulator columns.  skip_mma: issue no MMA
// so that the kernel's bounded wait runs out and sets *err.
cudaError_t launch_rate_gemm_probe(const float2* y, const float2* tw_m, int M, int l, int precision, int skip_mma,
                                   float* out, unsigned int* err, cudaStream_t s);
cudaError_t launch_select_batch(Batch& b, cudaStream_t s, int* n_launch);
cudaError_t launch_match_batch(Batch& b, cudaStream_t s, int* n_launch);
// Single-range search, one CTA per unit (used where no counter may be
// allocated).
cudaError_t launch_search(const SearchArgs& a, int pad_rate, cudaStream_t s, int* n_launch);

}  // namespace vk
