// Throughput probes for the roofline denominators the measured peak file does not give: the FP64
// and FP32 FMA rates of the SMs, and the dense rates of this library's tcgen05 grouped GEMM in bf16
// and tf32 on one 8192^3 problem.  All timed with CUDA events on the caller's stream.
#include <vector>

#include "plans.h"

namespace pd {
dmrg_status fail(const Error& e);

namespace {

// Eight independent FMA chains per thread (enough to hide the pipe latency); the result is
// written only when it is impossible, so the chains are not removed.
template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == T(-12345.0)) out[blockIdx.x] = s;
}

// Deterministic operand fill in (-1, 1): a hashed pattern, so the tensor cores see varied data.
template <class T>
__global__ void k_probe_fill(T* __restrict__ p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)(i * 2654435761ull) ^ 0x9e3779b9u;
        h ^= h >> 15;
        h *= 0x85ebca6bu;
        h ^= h >> 13;
        p[i] = T((float)(h & 0xffff) / 32768.0f - 1.0f);
    }
}

template <class T>
double fma_rate(int sms, cudaStream_t st) {
    DBuf out;
    out.ensure(4096 * sizeof(T), st);
    const int blocks = sms * 8, threads = 256;
    const int iters = sizeof(T) == 8 ? 2000 : 40000;
    k_fma_probe<T><<<blocks, threads, 0, st>>>(out.as<T>(), iters / 10, T(0.9999999), T(1e-7));   // warm-up
    PD_LAUNCHED();
    cudaEvent_t e0, e1;
    PD_CK(cudaEventCreate(&e0));
    PD_CK(cudaEventCreate(&e1));
    PD_CK(cudaEventRecord(e0, st));
    k_fma_probe<T><<<blocks, threads, 0, st>>>(out.as<T>(), iters, T(0.9999999), T(1e-7));
    PD_LAUNCHED();
    PD_CK(cudaEventRecord(e1, st));
    PD_CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    PD_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    return flops / (ms * 1e-3) / 1e12;
}

double gemm_rate(Num t, cudaStream_t st) {
    const int n = 8192;
    const long long nn = (long long)n * n;
    DBuf A, B, C, err;
    A.ensure(nn * num_size(t), st);
    B.ensure(nn * num_size(t), st);
    C.ensure(nn * 4, st);
    err.ensure(4, st);
    PD_CK(cudaMemsetAsync(err.p, 0, 4, st));
    if (t == Num::BF16) {
        k_probe_fill<__nv_bfloat16><<<1024, 256, 0, st>>>(A.as<__nv_bfloat16>(), nn);
        k_probe_fill<__nv_bfloat16><<<1024, 256, 0, st>>>(B.as<__nv_bfloat16>(), nn);
    } else {
        k_probe_fill<float><<<1024, 256, 0, st>>>(A.as<float>(), nn);
        k_probe_fill<float><<<1024, 256, 0, st>>>(B.as<float>(), nn);
    }
    PD_LAUNCHED();
    GemmBatch g;
    g.add(n, n, 0, n, 1, n, 1, 1, n, {GSeg{0, 0, n, 0}});
    const int saved = g_prof_class;
    g_prof_class = PROF_NONE;
    run_gemm_tc(g, t, A.p, n, n, B.p, n, n, C.p, Num::F32, err.as<unsigned>(), st);   // warm-up
    cudaEvent_t e0, e1;
    PD_CK(cudaEventCreate(&e0));
    PD_CK(cudaEventCreate(&e1));
    const int reps = 5;
    PD_CK(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) run_gemm_tc(g, t, A.p, n, n, B.p, n, n, C.p, Num::F32, err.as<unsigned>(), st);
    PD_CK(cudaEventRecord(e1, st));
    PD_CK(cudaEventSynchronize(e1));
    g_prof_class = saved;
    float ms = 0.f;
    PD_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    unsigned h = 0;
    PD_CK(cudaMemcpy(&h, err.p, 4, cudaMemcpyDeviceToHost));
    PD_REQUIRE(!(h & ERRBIT_TIMEOUT), DMRG_ERR_TIMEOUT, "tensor-core probe timed out");
    return 2.0 * n * (double)n * n * reps / (ms * 1e-3) / 1e12;
}

}  // namespace

}  // namespace pd

using namespace pd;

extern "C" dmrg_status dmrg_probe(int kind, double* tflops_out, void* stream) {
    try {
        PD_REQUIRE(tflops_out && kind >= 0 && kind <= 3, DMRG_ERR_ARG, "probe kind must be 0..3");
        cudaStream_t st = (cudaStream_t)stream;
        int dev = 0, sms = 0;
        PD_CK(cudaGetDevice(&dev));
        PD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (kind >= 2) PD_REQUIRE(tc_available(), DMRG_ERR_STATE, "tensor-core probes need sm_103 tensor cores");
        switch (kind) {
            case 0: *tflops_out = fma_rate<double>(sms, st); break;
            case 1: *tflops_out = fma_rate<float>(sms, st); break;
            case 2: *tflops_out = gemm_rate(Num::BF16, st); break;
            default: *tflops_out = gemm_rate(Num::F32, st); break;
        }
        PD_CK(cudaStreamSynchronize(st));
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(e);
    }
}
