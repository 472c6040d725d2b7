// Host-side state of one segment's search, shared by the single-segment
// entry points (volks_api.cu) and batch plans (volks_plan.cu).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "volks_internal.h"

namespace vk {

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int validate(const volks_segment* s, const volks_params* p);
bool is_device_pointer(const void* p);
// a1 (see volks_shift_table in volks.h)
int shift_table(double f_lo_mhz, double chan_bw_mhz, int n_f, double t_ap_s, int n_ap, double dm_lo,
                double dm_step, int n_dm, int32_t* shifts, int32_t* nvalid);
// a10 (see volks_cross_match in volks.h)
std::vector<volks_candidate> cross_match(std::vector<volks_candidate> all, int min_baselines);
// Number of SMs of the current device.
int sm_count();

struct SegJob {
  volks_segment seg{};
  volks_params prm{};
  int seg_id = 0;
  int n_f = 0, M = 0, n_eff = 0, n_tiles = 0, n_tchunk = 0, tchunk = 1024, win_mask = 0;
  int prec = 0;              // effective precision of the rate search (effective_precision)
  int n_pol = 1;             // polarisation products summed after calibration
  bool slide = false;        // sliding segments (stride 1)
  bool use_autos = false;    // HOPS normalisation with the stations' auto spectra
  int n_rows = 0;            // rows of the partial power sums: (pol, bl) or (pol, station)
  int win_log[kMaxWinLog + 1] = {}, win_off[kMaxWinLog + 1] = {}, word_off[kMaxWinLog + 1] = {};
  int win_off_l[kMaxWinLog + 1] = {};
  long long seg_per_bd = 0, word_per_bd = 0;
  int dm_chunk = 0;          // DM trials per range (the keys/bits buffers hold one chunk)
  bool empty = true;         // no work (n_bl * n_ap * n_dm == 0)
  std::vector<int32_t> shifts, nvalid;
  std::vector<double2> h_phasor;   // [n_pol][n_bl][n_f]
  std::vector<int2> h_blst;
  std::vector<float2> h_tw_n, h_tw_m;
  // device buffers
  const float2* d_vis = nullptr;
  void* d_vis_copy = nullptr;
  const float* d_autos = nullptr;
  void* d_autos_copy = nullptr;
  int2* d_blst = nullptr;
  float2* d_xn = nullptr;
  double* d_part = nullptr;
  double2* d_phasor = nullptr;
  float2* d_gain = nullptr;
  int32_t* d_shifts = nullptr;
  int32_t* d_nvalid = nullptr;
  float2* d_tw_n = nullptr;
  float2* d_tw_m = nullptr;
  unsigned long long* d_keys = nullptr;
  double* d_stats = nullptr;
  uint32_t* d_bits = nullptr;
  DevCand* d_cand = nullptr;
  unsigned int* d_count = nullptr;
  unsigned int cap = 0;
  bool stream_ordered = false;

  // Host tables (shift table, phasor, twiddles); dm_chunk <= 0: all DMs.
  int init(const volks_segment& s, const volks_params& p, int dm_chunk);
  int n_chunks() const { return empty ? 0 : (prm.n_dm + dm_chunk - 1) / dm_chunk; }
  // Device bytes the buffers need (input copy excluded).
  size_t device_bytes() const;
  // Bytes of the borrowed input (vis, plus auto spectra when used).
  size_t input_bytes() const;
  size_t keys_bytes_per_dm() const { return (size_t)seg.n_bl * seg_per_bd * 8; }
  // Allocate every buffer (stream-ordered on s, or plain cudaMalloc).
  int alloc(cudaStream_t s, bool stream_ordered_alloc);
  // Copy vis to the device when it is host memory (stream-ordered copy).
  int stage_input(cudaStream_t s);
  // Tables to the device (async on s from the job's host vectors).
  int upload(cudaStream_t s);
  void release(cudaStream_t s);
  // Descriptor of DM chunk c (base left 0).
  SegDesc desc(int c) const;
  // a2-a3 launches.
  cudaError_t enqueue_prep(cudaStream_t s, int* n_launch) const;
};

}  // namespace vk
