// Internal declarations shared by the host driver (volks_api.cu) and the
// kernels (volks_kernels.cu).  Not part of the ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vk {

constexpr int kTile = 32;          // APs per search tile (largest window)
constexpr int kMaxWinLog = 5;      // windows 1, 2, 4, 8, 16, 32
constexpr int kMaxSegPerTile = 63; // 32 + 16 + 8 + 4 + 2 + 1

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

struct PrepArgs {
  const float2* vis;               // [n_bl][n_ap][n_f]
  float2* xn;                      // [n_bl][n_f][n_ap]  (normalised, calibrated)
  double* part;                    // [n_bl][n_tchunk][n_f] partial sums of |S|^2
  const double2* phasor;           // [n_bl][n_f] calibration phasor (FP64)
  float2* gain;                    // [n_bl][n_f]
  int n_bl, n_ap, n_f, n_chan, n_tchunk, tchunk;
  int normalize, skip_first_chan;
};

struct SearchArgs {
  const float2* xn;                // [n_bl][n_f][n_ap]
  const int32_t* shifts;           // [n_dm][n_f]
  const int32_t* nvalid;           // [n_dm]
  const float2* tw_n;              // W_N^i, i < N   (N = n_f per residue pass)
  const float2* tw_m;              // W_M^i, i < M   (M = pad_delay * n_f)
  unsigned long long* keys;        // [n_bl][n_dm][seg_per_bd]
  int n_bl, n_ap, n_f, n_dm, pad_delay, M;
  int win_mask;                    // bit l set: window 2^l searched
  int win_off[kMaxWinLog + 1];     // segment offset of window 2^l inside a (b, d) block
  long long seg_per_bd;
  int n_tiles;
  int fold;                        // n_f = 512 only: 1 = one 512-thread CTA, else two 256-thread CTAs
};

struct SelectArgs {
  const unsigned long long* keys;
  const int32_t* nvalid;
  double* stats;                   // [n_bl][n_dm][n_win][2] mean, std
  uint32_t* bits;                  // [n_bl][n_dm][word_per_bd]
  int n_bl, n_dm, n_win, n_eff;
  int win_log[kMaxWinLog + 1];     // log2 of window i
  int win_off[kMaxWinLog + 1];     // segment offset of window i in a (b, d) block
  int word_off[kMaxWinLog + 1];    // bit-word offset of window i in a (b, d) block
  long long seg_per_bd, word_per_bd;
  double thresh;
};

struct MatchArgs {
  const unsigned long long* keys;
  const double* stats;
  const uint32_t* bits;
  const int32_t* nvalid;
  DevCand* out;
  unsigned int* count;
  unsigned int cap;
  int n_bl, n_dm, n_win, n_eff, min_windows;
  int win_log[kMaxWinLog + 1];
  int win_off[kMaxWinLog + 1];
  int word_off[kMaxWinLog + 1];
  long long seg_per_bd, word_per_bd;
};

// Set the calling thread's message returned by volks_last_error().
void set_last_error(const char* msg);

// Launchers (return the launch's cudaError_t).
cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s, int* n_launch);
cudaError_t launch_search(const SearchArgs& a, int pad_rate, cudaStream_t s, int* n_launch);
cudaError_t launch_select(const SelectArgs& a, cudaStream_t s, int* n_launch);
cudaError_t launch_match(const MatchArgs& a, cudaStream_t s, int* n_launch);

}  // namespace vk
