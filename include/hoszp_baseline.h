/*
 * hoszp_baseline.h — float32 operators of the traditional workflow
 * (Sec. IV-B and Fig. 4a: fully decompress, operate on the floats, fully
 * recompress), used as the comparator of the homomorphic operators. Together
 * with hoszp_decompress and hoszp_compress they form the GPU
 * "decompress -> op -> recompress" baseline. Same conventions as hoszp.h:
 * device pointers owned by the caller, asynchronous on `stream`, host-checkable
 * argument errors returned as HOSZP_ERR_ARG.
 */
#ifndef HOSZP_BASELINE_H
#define HOSZP_BASELINE_H

#include "hoszp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* y[i] = a * x[i] + b for i < n (negation: a = -1, b = 0; scalar addition:
 * a = 1, b = s; scalar multiplication: a = s, b = 0). y may equal x. Both
 * pointers 16-byte aligned. */
int hoszp_fop_axpb(const float* d_x, float* d_y, uint64_t n, float a, float b,
                   hoszp_stream_t stream);

/* z[i] = x[i] + y[i] (element-wise addition of two decompressed fields). */
int hoszp_fop_add(const float* d_x, const float* d_y, float* d_z, uint64_t n,
                  hoszp_stream_t stream);

/* Mean (variance = 0) or population variance (variance = 1) of n floats into
 * the device double *d_result: per-thread float32 partial sums of x and x^2,
 * combined in FP64. n >= 1. */
int hoszp_fop_moments(hoszp_ctx* ctx, const float* d_x, uint64_t n, int variance,
                      double* d_result, hoszp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HOSZP_BASELINE_H */
