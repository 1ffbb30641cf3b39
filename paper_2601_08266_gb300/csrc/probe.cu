// probe.cu -- measurement helper: the device's sustained FP32 / FP64 FMA rate
// on the CUDA cores, used as the ALU roofline of the VMS operators (which are
// bound by plain floating-point arithmetic, not by memory or tensor cores).
#include "fsi_internal.cuh"

namespace fsi {
namespace {

template <typename T> __global__ void fma_peak_kernel(int iters, T *out)
{
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    const T b = T(0.999999), c = T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == T(-12345.0)) out[blockIdx.x] = s;  // never true; keeps the chains live
}

template <typename T> fsi_status run(int device, double *rate)
{
    FSI_DEVICE(device);
    cudaDeviceProp prop;
    FSI_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    const int threads = 256, blocks = prop.multiProcessorCount * 8;
    T *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fsi_status st = check_cuda(cudaMalloc(&out, blocks * sizeof(T)), "probe buffer");
    if (st == FSI_OK) st = check_cuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    if (st == FSI_OK) st = check_cuda(cudaEventCreate(&e0), "event");
    if (st == FSI_OK) st = check_cuda(cudaEventCreate(&e1), "event");
    double best = 0.0;
    // iterations sized so that one launch runs for tens of milliseconds
    int iters = sizeof(T) == 8 ? 256 : 8192;
    for (int rep = 0; st == FSI_OK && rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        fma_peak_kernel<T><<<blocks, threads, 0, s>>>(iters, out);
        cudaEventRecord(e1, s);
        st = check_cuda(cudaEventSynchronize(e1), "probe kernel");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 0 && ms < 20.f && ms > 0.f) {  // scale up once, then measure
            iters = (int)(iters * (40.0 / ms));
            continue;
        }
        const double flops = 2.0 * 32.0 * iters * (double)threads * blocks;
        if (ms > 0.f && flops / (ms * 1e-3) > best) best = flops / (ms * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    if (st == FSI_OK) *rate = best;
    return st;
}

}  // namespace
}  // namespace fsi

extern "C" {

/* Declared in include/fsi.h. */
fsi_status fsi_measure_fma_peak(int device, fsi_prec prec, double *flops_per_second)
{
    if (!flops_per_second) return fsi::set_error(FSI_ERR_ARG, "NULL output");
    if (prec == FSI_F64) return fsi::run<double>(device, flops_per_second);
    if (prec == FSI_F32) return fsi::run<float>(device, flops_per_second);
    return fsi::set_error(FSI_ERR_ARG, "bad precision");
}

}  // extern "C"
