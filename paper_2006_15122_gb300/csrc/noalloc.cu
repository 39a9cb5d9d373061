// lattice_energies_noalloc: volume-averaged energies and means of scalar fields
// that the caller owns, computed without any device allocation.
//
// Some callers cannot allocate device memory: host programs that manage every
// byte of the GPU themselves (a simulation code with its own memory pool that has
// already claimed the device, a real-time loop that must never enter the
// allocator, a plug-in whose host owns the device).  This entry point takes
// their device arrays as they are and keeps its only scratch -- per-block partial
// sums and a completion counter -- in a fixed file-scope device array, so a call
// needs no cudaMalloc, cudaFree or allocating library routine.
//
// Scratch: CL_NOALLOC_MAX_BLOCKS blocks x 16 partial sums (FP64) plus a counter,
// about 128 KiB, held by every GPU that loads the library until the process exits.
// All calls share it and it keeps the last call's contents; the counter is cleared
// at the start of every call.  Two calls that overlap on the GPU (different streams,
// or different host threads on one device) race on it.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "cl_internal.cuh"

namespace {

constexpr int kSums = 16;

struct NoAllocScratch {
    double partials[CL_NOALLOC_MAX_BLOCKS * kSums];
    unsigned int counter;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device, looked up once per device with
// that device current (the host-side symbol is only a stand-in, never a device address).
constexpr int kMaxDevices = 64;
NoAllocScratch* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

struct NoAllocArgs {
    const double* phi;
    const double* pi;
    double* out;
    NoAllocScratch* scratch;
    int N, nf, pexp;
    double lam, q, idx2, a;
};

// One thread per site (grid-stride): sums of phi - r, (phi - r)^2, pi^2, (D^+ phi)^2
// per field and of the two potential terms; the last block to finish reduces the
// partials in a fixed order and writes E_K, E_G, E_V, means and variances (section
// 4.4.1).  The shift r is the field's value at site 0: a field that is a large
// homogeneous value plus small fluctuations then keeps the digits of its variance,
// which <phi^2> - <phi>^2 of the full field would cancel away.
__global__ void energies_noalloc_kernel(const NoAllocArgs A) {
    const int N = A.N;
    const size_t n3 = (size_t)N * N * N;
    double s[kSums];
#pragma unroll
    for (int k = 0; k < kSums; ++k) s[k] = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
        const size_t ix = ((size_t)z * N + y) * N + (x + 1 == N ? 0 : x + 1);
        const size_t iy = ((size_t)z * N + (y + 1 == N ? 0 : y + 1)) * N + x;
        const size_t iz = ((size_t)(z + 1 == N ? 0 : z + 1) * N + y) * N + x;
        double f[2] = {0.0, 0.0};
        for (int c = 0; c < A.nf; ++c) {
            const double* F = A.phi + (size_t)c * n3;
            const double* P = A.pi + (size_t)c * n3;
            const double v = F[i], p = P[i], d = v - __ldg(F);
            const double gx = F[ix] - v, gy = F[iy] - v, gz = F[iz] - v;
            f[c] = v;
            s[4 * c + 0] += d;
            s[4 * c + 1] += d * d;
            s[4 * c + 2] += p * p;
            s[4 * c + 3] += gx * gx + gy * gy + gz * gz;
        }
        double ap = 1.0;
        for (int k = 0; k < A.pexp; ++k) ap *= fabs(f[0]);
        s[8] += A.lam / A.pexp * ap;
        if (A.nf > 1) s[9] += 0.5 * A.q * f[0] * f[0] * f[1] * f[1];
    }
    __shared__ double red[32][kSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < kSums; ++k) {
        const double v = cl::warp_sum(s[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += red[w][threadIdx.x];
        A.scratch->partials[(size_t)blockIdx.x * kSums + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int last;
    if (threadIdx.x == 0) last = (atomicAdd(&A.scratch->counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[kSums];
    if (threadIdx.x < kSums) {
        double ks = 0.0, kc = 0.0;  // Kahan, fixed block order
        for (unsigned b = 0; b < gridDim.x; ++b) {
            const double xv = __ldcg(&A.scratch->partials[(size_t)b * kSums + threadIdx.x]);
            const double yk = xv - kc, tk = ks + yk;
            kc = (tk - ks) - yk;
            ks = tk;
        }
        tot[threadIdx.x] = (ks - kc) / (double)n3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double a2 = A.a * A.a, a6 = a2 * a2 * a2;
        for (int c = 0; c < 2; ++c) {
            const bool on = c < A.nf;
            const double r = on ? A.phi[(size_t)c * n3] : 0.0;  // the shift of the sums
            A.out[c] = on ? tot[4 * c + 2] / (2.0 * a6) : 0.0;                 // E_K
            A.out[2 + c] = on ? tot[4 * c + 3] * A.idx2 / (2.0 * a2) : 0.0;    // E_G
            A.out[6 + c] = on ? r + tot[4 * c + 0] : 0.0;                      // <phi>
            A.out[8 + c] = on ? tot[4 * c + 1] - tot[4 * c + 0] * tot[4 * c + 0] : 0.0;  // variance
        }
        A.out[4] = tot[8];  // <(lam/p)|phi|^p>
        A.out[5] = tot[9];  // <(q/2) phi^2 chi^2>
        A.scratch->counter = 0u;
    }
}

}  // namespace

namespace cl {
void set_global_error(const char* msg);
}

namespace {
cl_status cuda_error(const char* where, cudaError_t e) {
    char msg[256];
    snprintf(msg, sizeof(msg), "lattice_energies_noalloc: %s: %s", where, cudaGetErrorString(e));
    cl::set_global_error(msg);
    return CL_ERR_CUDA;
}
}  // namespace

extern "C" cl_status lattice_energies_noalloc(const cl_model* model, int32_t N, double kIR, double a,
                                              const double* phi, const double* pi, double* out, void* cuda_stream) {
    if (!model || !phi || !pi || !out) {
        cl::set_global_error("lattice_energies_noalloc: model, phi, pi and out must be non-NULL");
        return CL_ERR_ARG;
    }
    if (model->kind != CL_MODEL_SCALAR || model->n_fields < 1 || model->n_fields > 2 ||
        (model->pexp != 2 && model->pexp != 4 && model->pexp != 6)) {
        cl::set_global_error("lattice_energies_noalloc: needs a scalar model with 1 or 2 fields and p in {2,4,6}");
        return CL_ERR_ARG;
    }
    if (N < 2 || N > CL_NOALLOC_MAX_N || !(kIR > 0) || !(a > 0)) {
        cl::set_global_error("lattice_energies_noalloc: N must lie in [2, 2048] (CL_NOALLOC_MAX_N), kIR and a > 0");
        return CL_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cl::set_global_error("lattice_energies_noalloc: no usable current CUDA device");
        return CL_ERR_CUDA;
    }
    NoAllocScratch* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cl::set_global_error("lattice_energies_noalloc: cudaGetSymbolAddress of the scratch array failed");
                return CL_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<NoAllocScratch*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    const size_t n3 = (size_t)N * N * N;
    long long grid = (long long)sms * 4;
    const long long need = (long long)((n3 + 255) / 256);
    if (grid > need) grid = need;
    if (grid > CL_NOALLOC_MAX_BLOCKS) grid = CL_NOALLOC_MAX_BLOCKS;
    // A launch error is read with cudaGetLastError, which also returns (and clears)
    // an error left pending by earlier, unrelated work on this thread; refuse to
    // start while one is pending, so that the status below is this call's own.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_error("a CUDA error from earlier work is pending", e);
    e = cudaMemsetAsync(&scratch->counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_error("clearing the scratch counter", e);
    NoAllocArgs A;
    A.phi = phi;
    A.pi = pi;
    A.out = out;
    A.scratch = scratch;
    A.N = N;
    A.nf = model->n_fields;
    A.pexp = model->pexp;
    A.lam = model->lam;
    A.q = model->q;
    const double dx = 2.0 * M_PI / (kIR * N);
    A.idx2 = 1.0 / (dx * dx);
    A.a = a;
    energies_noalloc_kernel<<<(unsigned)grid, 256, 0, s>>>(A);
    e = cudaGetLastError();
    return e == cudaSuccess ? CL_OK : cuda_error("launching the energies kernel", e);
}
