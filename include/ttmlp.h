/* Learned surrogate for the tensor-train pricer: the kernels of a small
 * multilayer perceptron (fully connected layers with SiLU), its training
 * (backward pass, Adam) and its ensemble inference.
 *
 * The paper has no learned component; it names a better starting point for
 * TT-cross at high dimension as open (Section VI).  Here a network maps option
 * parameters to the price the TT pricer computes, trained on prices that pricer
 * generates; quotes whose ensemble members disagree go back to the TT pricer.
 *
 * Conventions for every call:
 *  - all array arguments are DEVICE pointers, owned by the caller, row-major,
 *    FP32 unless the name says bf16 (IEEE bfloat16 bit patterns in uint16_t);
 *  - `stream` is a cudaStream_t (NULL = legacy default stream); calls only
 *    enqueue work and return TT_MLP_OK, or TT_MLP_INVALID for a bad size or a
 *    NULL pointer, or TT_MLP_CUDA when a launch fails;
 *  - a layer has `in` inputs and `out` outputs; its weight is W[out][in] and its
 *    bias b[out]; x is [batch][in], z and a are [batch][out].
 */
#ifndef TTMLP_H
#define TTMLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { TT_MLP_OK = 0, TT_MLP_INVALID = -1, TT_MLP_CUDA = -5 };
enum { TT_MLP_LINEAR = 0, TT_MLP_SILU = 1 };

/* z = x W^T + b; a = act(z) (a may equal z for TT_MLP_LINEAR). */
int tt_mlp_forward(const float* x, int batch, int in, const float* w, const float* b, int out, int act,
                   float* z, float* a, void* stream);

/* The same with bfloat16 weights (inference copy); products accumulate in FP32. */
int tt_mlp_forward_bf16(const float* x, int batch, int in, const uint16_t* w_bf16, const float* b, int out,
                        int act, float* z, float* a, void* stream);

/* Inference layer on the tensor cores (tcgen05.mma kind::f16): a = act(x W^T + b)
 * with x [batch][in] and W [out][in] in bfloat16 and FP32 accumulation; writes a
 * as FP32 (a, nullable) and/or rounded to bfloat16 (a_bf16, nullable; the next
 * layer's input).  Needs in and out multiples of 16, 16..256 (pad the input with
 * zero columns, W with zero columns to match).  A tile whose completion wait runs
 * out of its bound gets NaN. */
int tt_mlp_forward_tc(const uint16_t* x_bf16, int batch, int in, const uint16_t* w_bf16, const float* b, int out,
                      int act, float* a, uint16_t* a_bf16, void* stream);

/* Backward of one layer: g = da * act'(z) (da for TT_MLP_LINEAR), written over da
 * (da holds dL/da on entry and dL/dz on return); dw = g^T x and db = column sums
 * of g (both overwritten); dx = g W when dx != NULL. */
int tt_mlp_backward(const float* x, const float* z, float* da, int batch, int in, const float* w,
                    int out, int act, float* dx, float* dw, float* db, void* stream);

/* Mean squared error over n values: dy = 2 (y - t) / n, *loss = mean (y - t)^2. */
int tt_mlp_mse(const float* y, const float* t, int n, float* dy, float* loss, void* stream);

/* Adam (Kingma and Ba 2015), step number `step` >= 1, on n parameters p with
 * gradient g and moments m, v (updated in place). */
int tt_mlp_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float beta1, float beta2,
                float eps, int step, void* stream);

/* Round FP32 to bfloat16 (to nearest, ties to even). */
int tt_mlp_to_bf16(const float* src, uint16_t* dst, long long n, void* stream);

/* Ensemble statistics over E members' predictions preds[E][n]:
 * mean[i] = average, spread[i] = max - min. */
int tt_mlp_ensemble(const float* preds, int members, int n, float* mean, float* spread, void* stream);

/* rows of src gathered by idx: dst[i][:] = src[idx[i]][:] (minibatch shuffling). */
int tt_mlp_gather(const float* src, const int* idx, int rows, int cols, float* dst, void* stream);

#ifdef __cplusplus
}
#endif
#endif
