// fp64_rate.cu -- the FP64 issue rate of the GPU, measured: the denominator of
// the "alu" roofline of the FP64 stencil kernels (every one of them is bound
// by FP64 add / multiply / FMA issue, not by HBM, on this part).
//
// Every thread runs 8 independent FMA chains x <- x * a + b (a, b runtime
// values, so nothing folds); enough warps per SM hide the FMA latency, so the
// kernel time is set by the FP64 pipe's issue rate.  One FMA counts as one
// FP64 operation, as in the library's algorithmic operation counts.
#include <cuda_runtime.h>

#include "../../../include/isdc_probe.h"

namespace {

template <int CHAINS>
__global__ void __launch_bounds__(256) k_dfma_chains(int iters, double a, double b, double* __restrict__ sink) {
  double x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = 1e-3 * double(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == -1.0) sink[threadIdx.x] = s;  // never true for these inputs; keeps the chains live
}

template <int CHAINS>
void launch(int blocks, int iters, cudaStream_t st) {
  k_dfma_chains<CHAINS><<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7, nullptr);
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int isdc_probe_fp64_rate(double* ops_per_s, double* ms_best) {
  if (!ops_per_s) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return 2;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // shapes: 4, 8 or 16 chains per thread at 4, 8 or 16 blocks of 256 threads
  // per SM; about 10 G FMAs per launch; after a warm-up of about 0.3 s the
  // best rate over three rounds of every shape is the peak
  const int chains[3] = {4, 8, 16}, bps[3] = {4, 8, 16};
  float best = 1e30f;
  double best_ops = 0.0;
  int rc = 0;
  for (int round = 0; round < 4 && rc == 0; ++round)
    for (int ci = 0; ci < 3 && rc == 0; ++ci)
      for (int bi = 0; bi < 3 && rc == 0; ++bi) {
        const int blocks = sms * bps[bi], ch = chains[ci];
        const int iters = int(10e9 / (double(blocks) * 256.0 * ch));
        const double ops = double(blocks) * 256.0 * double(iters) * ch;
        cudaEventRecord(e0, st);
        if (ch == 4) launch<4>(blocks, iters, st);
        else if (ch == 8) launch<8>(blocks, iters, st);
        else launch<16>(blocks, iters, st);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          rc = 2;
        else if (round > 0 && ops / ms > best_ops / best) {
          best = ms;
          best_ops = ops;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (rc) return rc;
  *ops_per_s = best_ops / (double(best) * 1e-3);
  if (ms_best) *ms_best = best;
  return 0;
}
