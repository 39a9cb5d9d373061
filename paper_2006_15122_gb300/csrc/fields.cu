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

// The stored representation: array = stored - shift (in T, as the passes apply
// it), mean = the FP64 homogeneous value; field = mean + array.
template <typename T>
__global__ void get_stored_kernel(const T* src, T* dst, size_t n, const DevState* st, int kind, int comp) {
    T shift = T(0);
    if (kind == 1) shift = T(st->sphi[comp]);
    if (kind == 2) shift = T(st->spi[comp]);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i] - shift;
}

__global__ void read_mean_kernel(const DevState* st, int kind, int comp, double* out) {
    *out = kind == 1 ? st->phibar[comp] : kind == 2 ? st->pibar[comp] : 0.0;
}

__global__ void write_mean_kernel(DevState* st, int kind, int comp, double mean) {
    if (kind == 1) { st->phibar[comp] = mean; st->sphi[comp] = 0.0; }
    if (kind == 2) { st->pibar[comp] = mean; st->spi[comp] = 0.0; }
}

// Stored array of `slot` (pending shift applied) into dst, a device buffer of
// N^3 elements of the handle's precision; its mean into *mean_dev (device).
cudaError_t launch_get_stored(Lattice* L, int slot, void* dst, double* mean_dev, cudaStream_t s) {
    const size_t n = (size_t)L->mc.N * L->mc.N * L->mc.N;
    int kind, comp;
    slot_kind(L->mc, slot, &kind, &comp);
    const int grid = L->sm_count * 8;
    const void* src = L->buf.f[L->cur][slot];
    if (L->prec == CL_FP32)
        get_stored_kernel<float><<<grid, 256, 0, s>>>((const float*)src, (float*)dst, n, L->buf.st, kind, comp);
    else
        get_stored_kernel<double><<<grid, 256, 0, s>>>((const double*)src, (double*)dst, n, L->buf.st, kind, comp);
    read_mean_kernel<<<1, 1, 0, s>>>(L->buf.st, kind, comp, mean_dev);
    return cudaGetLastError();
}

// The array of `slot` is overwritten by the caller (a copy into
// L->buf.f[L->cur][slot]); this sets its mean and clears its pending shift.
cudaError_t launch_set_stored_mean(Lattice* L, int slot, double mean, cudaStream_t s) {
    int kind, comp;
    slot_kind(L->mc, slot, &kind, &comp);
    write_mean_kernel<<<1, 1, 0, s>>>(L->buf.st, kind, comp, mean);
    return cudaGetLastError();
}

int has_mean(const ModelConst& mc, int slot) {
    int kind, comp;
    slot_kind(mc, slot, &kind, &comp);
    return kind != 0;
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

// FFT of the FP64 work array and shell binning into L->bins (added when accumulate)
static cudaError_t spectrum_of_work(Lattice* L, int accumulate, cudaStream_t s) {
    const int N = L->mc.N;
    const int nbins = spectrum_bins(N);
    if (cufftExecD2Z(L->plan_r2c, L->work, (cufftDoubleComplex*)L->cwork) != CUFFT_SUCCESS) return cudaErrorUnknown;
    if (!accumulate) cudaMemsetAsync(L->bins, 0, 3 * (size_t)nbins * sizeof(double), s);
    const size_t smem = 3 * (size_t)nbins * sizeof(double);
    bin_kernel<<<L->sm_count * 2, 512, smem, s>>>((const double2*)L->cwork, N, nbins, L->bins);
    return cudaGetLastError();
}

// Magnetic field of the U(1) sector, component i (sections 5.4, 5.2):
// B_i = f(theta_jk(n))/(e dx^2) with (i, j, k) cyclic, theta_jk the plaquette
// angle, f = sin (compact: B_i = -Im V_jk/(e dx^2)) or the identity (non-compact:
// B_i = eps_ijk D_j^+ A_k).
template <typename T>
__global__ void u1_magnetic_kernel(const T* tj, const T* tk, int N, int j, int k, double c, int nc, double* out) {
    const size_t n3 = (size_t)N * N * N;
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < n3; n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / ((size_t)N * N));
        const int c0[3] = {x, y, z};
        int pj[3] = {x, y, z}, pk[3] = {x, y, z};
        pj[j] = c0[j] + 1 == N ? 0 : c0[j] + 1;
        pk[k] = c0[k] + 1 == N ? 0 : c0[k] + 1;
        const size_t nj = ((size_t)pj[2] * N + pj[1]) * N + pj[0], nk = ((size_t)pk[2] * N + pk[1]) * N + pk[0];
        const double t = (double)tj[n] + (double)tk[nj] - (double)tj[nk] - (double)tk[n];
        out[n] = c * (nc ? t : sin(t));
    }
}

// Magnetic field of the SU(2) sector, component (i, a) (section 6.3):
// B_i^a = -2 q_a[U_jk(n)]/(g dx^2), (i, j, k) cyclic, U_jk = U_j(n) U_k(n+j) U_j^dag(n+k) U_k^dag(n)
// as a unit quaternion q0 + i q.sigma.
__device__ __forceinline__ void qmul_d(const double* p, const double* q, double* r) {
    const double r0 = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
    const double r1 = p[0] * q[1] + q[0] * p[1] - (p[2] * q[3] - p[3] * q[2]);
    const double r2 = p[0] * q[2] + q[0] * p[2] - (p[3] * q[1] - p[1] * q[3]);
    const double r3 = p[0] * q[3] + q[0] * p[3] - (p[1] * q[2] - p[2] * q[1]);
    r[0] = r0; r[1] = r1; r[2] = r2; r[3] = r3;
}
struct Links4 {
    const void* u[12];  // U_i component c at 4 i + c
};
template <typename T>
__global__ void su2_magnetic_kernel(Links4 U, int N, int j, int k, int a, double c, double* out) {
    const size_t n3 = (size_t)N * N * N;
    const T* const* u = reinterpret_cast<const T* const*>(U.u);
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < n3; n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / ((size_t)N * N));
        const int c0[3] = {x, y, z};
        int pj[3] = {x, y, z}, pk[3] = {x, y, z};
        pj[j] = c0[j] + 1 == N ? 0 : c0[j] + 1;
        pk[k] = c0[k] + 1 == N ? 0 : c0[k] + 1;
        const size_t nj = ((size_t)pj[2] * N + pj[1]) * N + pj[0], nk = ((size_t)pk[2] * N + pk[1]) * N + pk[0];
        double Uj[4], Ukj[4], Ujk[4], Uk[4], t1[4], t2[4], P[4];
        for (int q = 0; q < 4; ++q) {
            const double sg = q == 0 ? 1.0 : -1.0;
            Uj[q] = (double)u[4 * j + q][n];
            Ukj[q] = (double)u[4 * k + q][nj];
            Ujk[q] = sg * (double)u[4 * j + q][nk];  // U_j^dag(n+k)
            Uk[q] = sg * (double)u[4 * k + q][n];    // U_k^dag(n)
        }
        qmul_d(Uj, Ukj, t1);
        qmul_d(t1, Ujk, t2);
        qmul_d(t2, Uk, P);
        out[n] = c * P[1 + a];
    }
}

cudaError_t launch_gauge_spectrum(Lattice* L, int sector, int what, int* ncomp, cudaStream_t s) {
    const int N = L->mc.N;
    const int grid = L->sm_count * 8;
    const size_t n3 = (size_t)N * N * N;
    cudaError_t e = cudaSuccess;
    int nc = 0;
    void** b = L->buf.f[L->cur];
    if (sector == 0) {  // U(1): angles and electric momenta
        const int th = L->mc.kind == CL_MODEL_U1 ? 4 : 29, ea = L->mc.kind == CL_MODEL_U1 ? 7 : 32;
        const double eg = L->mc.kind == CL_MODEL_U1 ? L->mc.e : L->mc.e2;
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
            if (what == 0) {
                e = launch_get_field(L, ea + i, L->work, s);
            } else {
                const int j = (i + 1) % 3, k = (i + 2) % 3;
                const double c = 1.0 / (eg * L->mc.dx * L->mc.dx);
                if (L->prec == CL_FP32)
                    u1_magnetic_kernel<float><<<grid, 256, 0, s>>>((const float*)b[th + j], (const float*)b[th + k], N, j, k,
                                                                   c, L->mc.nc, L->work);
                else
                    u1_magnetic_kernel<double><<<grid, 256, 0, s>>>((const double*)b[th + j], (const double*)b[th + k], N,
                                                                    j, k, c, L->mc.nc, L->work);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = spectrum_of_work(L, i > 0, s);
            ++nc;
        }
    } else {  // SU(2): links 8 + 4 i + c, electric momenta 20 + 3 i + a
        Links4 U;
        for (int q = 0; q < 12; ++q) U.u[q] = b[8 + q];
        for (int i = 0; i < 3 && e == cudaSuccess; ++i)
            for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
                if (what == 0) {
                    e = launch_get_field(L, 20 + 3 * i + a, L->work, s);
                } else {
                    const int j = (i + 1) % 3, k = (i + 2) % 3;
                    const double c = -2.0 / (L->mc.e * L->mc.dx * L->mc.dx);
                    if (L->prec == CL_FP32) su2_magnetic_kernel<float><<<grid, 256, 0, s>>>(U, N, j, k, a, c, L->work);
                    else su2_magnetic_kernel<double><<<grid, 256, 0, s>>>(U, N, j, k, a, c, L->work);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess) e = spectrum_of_work(L, nc > 0, s);
                ++nc;
            }
    }
    (void)n3;
    *ncomp = nc;
    return e;
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

// cuTensorMapEncodeTiled, resolved once through the runtime (no link against the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn tensor_map_encoder() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        const bool ok = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                            cudaSuccess &&
                        q == cudaDriverEntryPointSuccess;
        cudaGetLastError();
        return ok ? reinterpret_cast<EncodeTiledFn>(p) : nullptr;
    }();
    return fn;
}

bool encode_plane_box(CUtensorMap* map, const void* base, int N, size_t tsize, int bx, int by) {
    const EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t n = (cuuint64_t)N;
    const cuuint64_t dims[3] = {n, n, n};
    const cuuint64_t strides[2] = {n * tsize, n * n * tsize};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t unit[3] = {1, 1, 1};
    const CUtensorMapDataType dt = tsize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, unit, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace cl
