// FP64 throughput probes (include/cardiac_gb300_measure.h).
#include <cstdio>
#include <string>

#include "cardiac_gb300_measure.h"
#include "cg_internal.h"

#define CG_API extern "C" __attribute__((visibility("default")))

namespace {

template <int OP>
__global__ void __launch_bounds__(256) k_fp64_rate(double *out, int64_t iters, double seed)
{
    // the one-lane variant: every lane but the first of each warp leaves
    if (OP == CG_MEASURE_DFMA_ONE_LANE && (threadIdx.x & 31) != 0) return;
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + 1e-7 * threadIdx.x + 1e-3 * i;
    const double b = 0.9999999, c = 1e-9;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == CG_MEASURE_DFMA || OP == CG_MEASURE_DFMA_ONE_LANE) a[i] = fma(a[i], b, c);
            if (OP == CG_MEASURE_DADD) a[i] = a[i] + c;
            if (OP == CG_MEASURE_DMUL) a[i] = a[i] * b;
            if (OP == CG_MEASURE_TANH) a[i] = fma(tanh(a[i]), 1.5, c);
            if (OP == CG_MEASURE_EXP) a[i] = fma(exp(-a[i]), 0.9, c);
            if (OP == CG_MEASURE_DIV) a[i] = b / a[i] + c;
        }
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 1.2345678) out[0] = s;   // keeps the chains live; never true in practice
}

thread_local std::string g_merr;

}  // namespace

CG_API cg_status cg_measure_fp64_rate(int32_t op, int64_t iters, double *ops_per_s, double *seconds)
{
    const void *k = nullptr;
    int64_t def = 0;
    switch (op) {
    case CG_MEASURE_DFMA: k = (const void *)&k_fp64_rate<CG_MEASURE_DFMA>; def = 40960; break;
    case CG_MEASURE_DADD: k = (const void *)&k_fp64_rate<CG_MEASURE_DADD>; def = 40960; break;
    case CG_MEASURE_DMUL: k = (const void *)&k_fp64_rate<CG_MEASURE_DMUL>; def = 40960; break;
    case CG_MEASURE_TANH: k = (const void *)&k_fp64_rate<CG_MEASURE_TANH>; def = 2048; break;
    case CG_MEASURE_EXP: k = (const void *)&k_fp64_rate<CG_MEASURE_EXP>; def = 2048; break;
    case CG_MEASURE_DIV: k = (const void *)&k_fp64_rate<CG_MEASURE_DIV>; def = 4096; break;
    case CG_MEASURE_DFMA_ONE_LANE: k = (const void *)&k_fp64_rate<CG_MEASURE_DFMA_ONE_LANE>; def = 40960; break;
    default: return CG_EINVAL;
    }
    if (iters <= 0) iters = def;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0;
    const int grid = sms * 4, block = 256;
    if (e == cudaSuccess) {
        double seed = 0.5;
        int64_t warm = iters / 2 + 1;
        void *wargs[] = {&out, &warm, &seed};
        e = cudaLaunchKernel(k, dim3(grid), dim3(block), wargs, 0, st);
        void *args[] = {&out, &iters, &seed};
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = cudaLaunchKernel(k, dim3(grid), dim3(block), args, 0, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        g_merr = cudaGetErrorString(e);
        return CG_ECUDA;
    }
    const double lanes = (op == CG_MEASURE_DFMA_ONE_LANE) ? (double)block / 32.0 : (double)block;
    const double nops = (double)grid * lanes * 8.0 * (double)iters;
    if (ops_per_s) *ops_per_s = nops / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3;
    return CG_OK;
}

// ------------------------------------------------ own elementary functions

#include <cmath>

#include "cg_fastmath.cuh"

namespace {

__global__ void k_check_fastmath(int fn, const double *x, double *own, double *ref, int64_t n, const double *tab)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        if (fn == 0) {
            own[i] = cgk::fast_rcp(v);
            ref[i] = 1.0 / v;
        } else if (fn == 1) {
            own[i] = cgk::exp_neg(v, tab);
            ref[i] = exp(v);
        } else {
            double ds;
            own[i] = cgk::sigmoid(v, tab, ds);
            ref[i] = 0.5 * (1.0 + tanh(0.5 * v));
        }
    }
}

}  // namespace

CG_API cg_status cg_check_fastmath(int32_t fn, const double *x, double *own, double *ref, int64_t n)
{
    if (fn < 0 || fn > 2 || !x || !own || !ref || n < 0) return CG_EINVAL;
    double tab[cgk::EXP_TAB];
    cgk::exp_table(tab, cgk::EXP_TAB);
    double *dtab = nullptr;
    cudaError_t e = cudaMalloc(&dtab, sizeof tab);
    if (e == cudaSuccess) e = cudaMemcpy(dtab, tab, sizeof tab, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_check_fastmath<<<1024, 256>>>(fn, x, own, ref, n, dtab);
        e = cudaDeviceSynchronize();
    }
    if (dtab) cudaFree(dtab);
    return e == cudaSuccess ? CG_OK : CG_ECUDA;
}
