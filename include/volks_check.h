/*
 * volks_check.h -- checking entry points of libvolks.so.
 *
 * These calls are not part of the search interface (include/volks.h): the
 * tests use them to pin internal layouts against independent computations
 * and to exercise fault paths without faulting the GPU.  They take the same
 * conventions as volks.h (return codes VOLKS_*, thread-local message in
 * volks_last_error()).
 */
#ifndef VOLKS_CHECK_H
#define VOLKS_CHECK_H

#include "volks.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Checking aid, outside the search: one 128-delay-cell block of the
 * tensor-core rate GEMM (Sec. 2.2 2-D search, Sec. 2.4.2 step 6 window
 * combine) of window `win` (2, 4, 8, 16 or 32 APs) at `precision` (VOLKS_BF16,
 * VOLKS_FP16 or VOLKS_FP8), through the same operand builders and MMA
 * issue as the search kernel, with operand scale 1.
 * y:   device complex64 [32][128] (APs x delay cells).
 * out: device float [128][256]; row c, column 8 win s + 2 q (+ 1) holds the
 *      real (imaginary) part of sum_{u < win} y[s win + u][c]
 *      exp(-2 pi i q u / (4 win)), q < 4 win, s < 32 / win, from y and the
 *      DFT coefficients rounded to the operand type, accumulated in FP32.
 * flags: VOLKS_CHECK_SKIP_MMA issues no MMA, so the kernel's bounded wait
 *      for the tensor cores (shortened to ~0.1 s here) runs out: the call
 *      must then return VOLKS_ETIMEOUT with the context still usable.
 * Synchronous (waits on the legacy default stream).  VOLKS_EINVAL for a
 * bad window, precision or flag, VOLKS_ETIMEOUT if the tensor cores did not
 * answer within the kernel's bounded wait, VOLKS_ECUDA otherwise.
 */
#define VOLKS_CHECK_SKIP_MMA 1
int volks_check_rate_gemm(const void *y, int32_t win, int32_t precision, int32_t flags, float *out);

/*
 * Checking accessor of the no-allocation variant (no paper counterpart):
 * copies the shift table (int32 [n_dm][n_f]) and n_valid (int32 [n_dm])
 * that the last volks_search_peaks_noalloc call on the current device
 * computed on the GPU into caller device buffers, on cuda_stream (device
 * to device copies; nothing is allocated).  n_dm and n_f must be the last
 * call's; VOLKS_EINVAL if they are not, if no call has run on the device,
 * or if a buffer is not device memory of the current device.  The copies
 * read the shared scratch, so they race with a later call that overlaps
 * them on the GPU.
 */
int volks_noalloc_tables(void *cuda_stream, int32_t *shifts, int32_t *nvalid, int32_t n_dm,
                         int32_t n_f);

#ifdef __cplusplus
}
#endif
#endif /* VOLKS_CHECK_H */
