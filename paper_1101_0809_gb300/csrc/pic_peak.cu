// pic_peak.cu -- pic_measure_fp64_fma: a kernel of independent FP64 fused
// multiply-add chains that fills the device, so that its duration gives the
// rate of FP64 FMA instructions, the unit that bounds the FP64 particle path.
#include "../../include/pic.h"
#include "pic_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(long long iters, double *sink)
{
    double a[kChains];
    const double m = 1.0 + 1e-12 * (threadIdx.x + 1), c = 1e-9 * blockIdx.x;
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = 1.0 + q * 1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == 12345.678) sink[0] = s;   // keeps the chains live; practically never taken
}

}  // namespace

extern "C" int pic_measure_fp64_fma(long long iters, int blocks_per_sm, double *sink, long long *fma_count,
                                    void *cuda_stream)
{
    if (iters <= 0 || blocks_per_sm <= 0 || !sink || !fma_count) {
        pic::set_last_error("pic_measure_fp64_fma: iters, blocks_per_sm > 0 and non-null sink, fma_count needed");
        return PIC_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        pic::set_last_error("pic_measure_fp64_fma: no device");
        return PIC_ERR_CUDA;
    }
    const long long blocks = (long long)sms * blocks_per_sm;
    k_fp64_fma<<<(unsigned)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(iters, sink);
    if (cudaGetLastError() != cudaSuccess) {
        pic::set_last_error("pic_measure_fp64_fma: launch failed");
        return PIC_ERR_CUDA;
    }
    *fma_count = blocks * 256 * iters * kChains;
    return PIC_OK;
}
