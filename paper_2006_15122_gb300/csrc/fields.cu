// Field transfer (mean + fluctuation <-> full FP64 field) and power spectra.
//
// Spectrum (sections 3.1, 4.4.2, 5.4.2): Delta(k) = k^3/(2 pi^2) (dx/N)^3
// <|f(n~)|^2>_R, the shell average taken over the modes with |n~| in
// [b, b+1) and k_b = k_IR times their mean |n~|.  |f(n~)|^2 does not depend
// on the sign convention of the transform, so cuFFT's D2Z serves; the R2C
// half space counts modes with 0 < n~_x < N/2 twice.
#include <math.h>

#include "cl_internal.cuh"

namespace cl {

int array_count(const ModelConst& mc) {
    if (mc.kind == CL_MODEL_SCALAR) return 2 * mc.nf;
    if (mc.kind == CL_MODEL_SU2) return mc.ext ? 37 : 29;
    return 10;
}

int array_slot(const ModelConst& mc, int which) {
    if (mc.kind == CL_MODEL_SCALAR) {
        if (which >= 0 && which < mc.nf) return which;
        if (which >= 4 && which < 4 + mc.nf) return mc.nf + which - 4;
        return -1;
    }
    if (mc.kind == CL_MODEL_SU2) {  // Phi 0-3, pi 4-7, links 16 + 4 i + c, piB 28 + 3 i + a
        if (which >= 0 && which < 8) return which;
        if (which >= 16 && which < 28) return which - 8;
        if (which >= 28 && which < 37) return which - 8;
        // U(1) angles 29-31, piA 32-34, chi 35, pchi 36
        if (mc.e2 > 0 && which >= 8 && which <= 10) return 29 + which - 8;
        if (mc.e2 > 0 && which >= 12 && which <= 14) return 32 + which - 12;
        if (mc.chi && (which == 37 || which == 38)) return 35 + which - 37;
        return -1;
    }
    if (which == 0 || which == 1) return which;
    if (which == 4 || which == 5) return which - 2;
    if (which >= 8 && which <= 10) return which - 4;
    if (which >= 12 && which <= 14) return which - 5;
    return -1;
}

// full = mean + (stored - shift), computed as the passes do: the subtraction in T, the sum in FP64
template <typename T>
__global__ void get_field_kernel(const T* src, double* dst, size_t n, const DevState* st, int kind, int comp) {
    double mean = 0.0;
    T shift = T(0);
    if (kind == 1) { mean = st->phibar[comp]; shift = T(st->sphi[comp]); }
    if (kind == 2) { mean = st->pibar[comp]; shift = T(st->spi[comp]); }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = mean + (double)(src[i] - shift);
}

__global__ void sum_kernel(const double* src, size_t n, double* partials) {
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        s += src[i];
    s = warp_sum(s);
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += w[k];
        partials[blockIdx.x] = t;
    }
}

__global__ void set_mean_kernel(const double* partials, int nblocks, size_t n, DevState* st, int kind, int comp) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[b];
    const double mean = t / (double)n;
    if (kind == 1) { st->phibar[comp] = mean; st->sphi[comp] = 0.0; }
    if (kind == 2) { st->pibar[comp] = mean; st->spi[comp] = 0.0; }
}

template <typename T>
__global__ void set_field_kernel(const double* src, T* dst, size_t n, const DevState* st, int kind, int comp) {
    double mean = 0.0;
    if (kind == 1) mean = st->phibar[comp];
    if (kind == 2) mean = st->pibar[comp];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = T(src[i] - mean);
}

// slot -> (kind: 0 plain, 1 field with mean, 2 momentum with mean; component)
static void slot_kind(const ModelConst& mc, int slot, int* kind, int* comp) {
    *kind = 0;
    *comp = 0;
    if (mc.kind == CL_MODEL_SCALAR) {
        if (slot < mc.nf) { *kind = 1; *comp = slot; }
        else { *kind = 2; *comp = slot - mc.nf; }
    }
}

cudaError_t launch_get_field(Lattice* L, int slot, double* dst, cudaStream_t s) {
    const size_t n = (size_t)L->mc.N * L->mc.N * L->mc.N;
    int kind, comp;
    slot_kind(L->mc, slot, &kind, &comp);
    const int grid = L->sm_count * 8;
    const void* src = L->buf.f[L->cur][slot];
    if (L->prec == CL_FP32) get_field_kernel<float><<<grid, 256, 0, s>>>((const float*)src, dst, n, L->buf.st, kind, comp);
    else get_field_kernel<double><<<grid, 256, 0, s>>>((const double*)src, dst, n, L->buf.st, kind, comp);
    return cudaGetLastError();
}

cudaError_t launch_set_field(Lattice* L, int slot, const double* src, cudaStream_t s) {
    const size_t n = (size_t)L->mc.N * L->mc.N * L->mc.N;
    int kind, comp;
    slot_kind(L->mc, slot, &kind, &comp);
    const int grid = L->sm_count * 4;
    if (kind != 0) {
        sum_kernel<<<grid, 256, 0, s>>>(src, n, L->buf.partials);
        set_mean_kernel<<<1, 1, 0, s>>>(L->buf.partials, grid, n, L->buf.st, kind, comp);
    }
    void* dst = L->buf.f[L->cur][slot];
    if (L->prec == CL_FP32) set_field_kernel<float><<<grid, 256, 0, s>>>(src, (float*)dst, n, L->buf.st, kind, comp);
    else set_field_kernel<double><<<grid, 256, 0, s>>>(src, (double*)dst, n, L->buf.st, kind, comp);
    return cudaGetLastError();
}

int spectrum_bins(int N) {
    const long long half = N / 2, n2 = 3 * half * half;
    long long r = (long long)sqrt((double)n2);
    while ((r + 1) * (r + 1) <= n2) ++r;
    while (r * r > n2) --r;
    return (int)(r + 1);
}

__device__ __forceinline__ int isqrt_exact(long long n2) {
    long long r = (long long)sqrt((double)n2);
    while ((r + 1) * (r + 1) <= n2) ++r;
    while (r * r > n2) --r;
    return (int)r;
}

// Shell sums of |F|^2, |n~| and the mode count; per-block shared histograms, then FP64 atomics.
__global__ void bin_kernel(const double2* F, int N, int nbins, double* out /* 3*nbins */) {
    extern __shared__ double h[];
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) h[i] = 0.0;
    __syncthreads();
    const int NH = N / 2 + 1;
    const size_t total = (size_t)N * N * NH;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % NH);
        const int iy = (int)((i / NH) % N);
        const int iz = (int)(i / ((size_t)NH * N));
        const long long my = iy <= N / 2 ? iy : iy - N, mz = iz <= N / 2 ? iz : iz - N;
        const long long n2 = (long long)ix * ix + my * my + mz * mz;
        const int b = isqrt_exact(n2);
        const double w = (ix == 0 || ix == N / 2) ? 1.0 : 2.0;
        const double2 v = F[i];
        atomicAdd(&h[b], w * (v.x * v.x + v.y * v.y));
        atomicAdd(&h[nbins + b], w * sqrt((double)n2));
        atomicAdd(&h[2 * nbins + b], w);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x)
        if (h[i] != 0.0) atomicAdd(&out[i], h[i]);
}

cudaError_t launch_spectrum(Lattice* L, int slot, int accumulate, cudaStream_t s) {
    const int N = L->mc.N;
    const int nbins = spectrum_bins(N);
    cudaError_t e = launch_get_field(L, slot, L->work, s);
    if (e != cudaSuccess) return e;
    if (cufftExecD2Z(L->plan_r2c, L->work, (cufftDoubleComplex*)L->cwork) != CUFFT_SUCCESS) return cudaErrorUnknown;
    if (!accumulate) cudaMemsetAsync(L->bins, 0, 3 * (size_t)nbins * sizeof(double), s);
    const size_t smem = 3 * (size_t)nbins * sizeof(double);
    bin_kernel<<<L->sm_count * 2, 512, smem, s>>>((const double2*)L->cwork, N, nbins, L->bins);
    return cudaGetLastError();
}

}  // namespace cl
