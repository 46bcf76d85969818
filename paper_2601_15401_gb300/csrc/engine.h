// Host orchestration entry points (engine.cu).
#pragma once
#include "internal.h"
#include "plan.h"

namespace ckks {

size_t mul_k_ws_bytes(const Context &C, const Plan &P, int level, int B);
size_t mul2_ws_bytes(const Context &C, int level, int B);
size_t relin_ws_bytes(const Context &C, int n, int level, int B);
size_t rescale_ws_bytes(const Context &C, int polys, int level, int mu, int B);
size_t rotate_ws_bytes(const Context &C, int level, int B);
int run_rotate_ws(const Context &C, int B, int level, uint32_t g, LimbView in, LimbView out, const u64 *keys,
                  void *ws, size_t bytes, cudaStream_t st, cudaError_t &err);

int run_mul_k_ws(const Context &C, const Plan &P, int level, int B, const LimbView *in, LimbView out,
                 const u64 *keys, int t_max, void *ws, size_t bytes, cudaStream_t st, cudaError_t &err);
int run_relin_ws(const Context &C, int B, int n, int level, LimbView D, const u64 *keys, bool out_ntt, LimbView out,
                 void *ws, size_t bytes, cudaStream_t st, cudaError_t &err);
int run_rescale_ws(const Context &C, int B, int polys, int level, int mu, LimbView in, LimbView out, void *ws,
                   size_t bytes, cudaStream_t st, cudaError_t &err);
size_t rescale_alg1_ws_bytes(const Context &C, int polys, int level, int mu, int B);
int run_rescale_alg1_ws(const Context &C, int B, int polys, int level, int mu, LimbView in, LimbView out, void *ws,
                        size_t bytes, cudaStream_t st, cudaError_t &err);
int run_mul2_ws(const Context &C, int level, int B, LimbView a, LimbView b, LimbView out, const u64 *keys,
                void *ws, size_t bytes, cudaStream_t st, cudaError_t &err);
cudaError_t run_tensor(const Context &C, int B, int level, int m, const LimbView *in, const int *polys,
                       LimbView out, cudaStream_t st);
cudaError_t transform_plain(const Context &C, bool fwd, int B, int polys, int level, LimbView in, LimbView out,
                            cudaStream_t st);

// scale of a plan's output from the inputs' scales (Section V: each
// rescale divides by the prime it removes)
double plan_scale(const Context &C, const Plan &P, int level, const double *scales);

int context_build(Context &C, uint32_t log_n, uint32_t L, uint32_t K, uint32_t dnum, const u64 *q, const u64 *p,
                  int device);
void context_release(Context &C);

}  // namespace ckks
