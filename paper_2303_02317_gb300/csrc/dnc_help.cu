// dnc_help.cu -- the pricing kernels of batch launches whose CTAs help one
// another (board tasks and helping sessions), compiled apart from the plain
// kernels in dnc.cu so that both translation units build in parallel.  The
// FP32-split mode has no helping kernel.
#include "dnc_kernel.cuh"

namespace aop {

cudaError_t launch_dnc_help(int method, unsigned grid, int threads, size_t smem, cudaStream_t s,
                            const DncArgs &a) {
    switch (method) {
    case AOP_FFT_FP64:
        cudaFuncSetAttribute(dnc_kernel<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dnc_kernel<0, true><<<grid, threads, smem, s>>>(a);
        break;
    case AOP_FFT_DF32:
        cudaFuncSetAttribute(dnc_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dnc_kernel<2, true><<<grid, threads, smem, s>>>(a);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace aop
