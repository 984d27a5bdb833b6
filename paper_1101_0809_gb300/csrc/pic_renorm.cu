// pic_renorm.cu -- pic_renormalize_f32: the FP32 form's offset-to-cell
// renormalization (the move of Eq. coordscheme, Appendix step 2c) applied to
// caller-given (offset, displacement) pairs.  It runs the very device function
// the FP32 particle kernels call, so that its result can be checked bit for bit
// against a double-precision renormalization rounded once to float.
#include <cstdio>

#include "../../include/pic.h"
#include "pic_internal.h"

namespace {

__global__ void k_renormalize(long long n, const float *off, const float *delta, int *shift, float *out)
{
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    float o = 0.f;
    shift[p] = pic::renormalize(off[p], delta[p], o);
    out[p] = o;
}

int fail(int code, const char *m)
{
    pic::set_last_error(m);
    return code;
}

}  // namespace

extern "C" int pic_renormalize_f32(const float *offset, const float *delta, long long n, int *shift,
                                   float *offset_out, void *cuda_stream)
{
    if (n < 0 || n > (1LL << 40)) return fail(PIC_ERR_INVALID_ARG, "n out of range");
    if (n == 0) return PIC_OK;
    if (!offset || !delta || !shift || !offset_out) return fail(PIC_ERR_INVALID_ARG, "null array");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nthr = 256;
    k_renormalize<<<(unsigned)((n + nthr - 1) / nthr), nthr, 0, st>>>(n, offset, delta, shift, offset_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char m[160];
        snprintf(m, sizeof(m), "renormalize kernel launch: %s", cudaGetErrorString(e));
        return fail(e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA, m);
    }
    return PIC_OK;
}
