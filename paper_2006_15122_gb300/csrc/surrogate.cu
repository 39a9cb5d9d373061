// Surrogate multilayer perceptron on BF16 tensor cores (a workload pattern
// around the paper's method, not a part of the paper): maps (log10 q, t) to the
// lattice observables of an ensemble scan.
//
//   H_0 = X,  Z_l = H_l W_l^T + b_l,  H_{l+1} = GELU(Z_l),  Y = Z_L,
//   loss = mean (Y - T)^2,  GELU(x) = x/2 (1 + erf(x/sqrt 2)),
// trained by Adam on FP32 master weights; every GEMM (forward, input and
// weight gradients) runs on the fifth-generation tensor cores (tcgen05.mma with
// the accumulator in tensor memory) with BF16 operands and FP32 accumulation,
// the bias/GELU epilogues fused.
// Matrices are stored row-major with every dimension padded with zeros to a
// multiple of 32 (batch: 64), so that the GEMM needs no K-edge handling and the
// padding stays zero through forward and backward passes.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "cl_internal.cuh"

namespace cl {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------- GEMM
// C[M x N] = A[M x K] . B[N x K]^T  (A, B bf16 row-major; K a multiple of 32)
struct GemmArgs {
    const bf16* A;
    int lda;
    const bf16* B;
    int ldb;
    float* C;
    int ldc;
    int M, N, K;
    int mode;           // 0: C = acc;  1: C = Z = acc + bias, H = bf16(GELU(Z));  2: C = acc + bias;
                        // 3: C = dZ = acc GELU'(Zp), H = bf16(dZ) (the backward step through a hidden layer)
    const float* bias;  // length >= Nvalid
    bf16* H;
    int ldh;
    int Mvalid, Nvalid;  // outside: written as zero (keeps the padding zero)
    const float* Zp;     // mode 3: pre-activations of the layer below (M x N, leading dimension ldz)
    int ldz;
    bf16* HT;            // optional: the bf16 output transposed, HT[c * ldht + r]
    int ldht;
    float* cs;           // optional: sums over this CTA's rows of each column of C, cs[blockIdx.y * ldcs + c]
    int ldcs;
    int kchunk;          // K per split (a multiple of 64): CTA z of the grid sums K range [z kchunk, (z+1) kchunk)
    size_t cstride;      // and writes its partial C at C + z cstride (mode 0 only)
};

__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool valid) {
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime_f(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// ---------------------------------------------------------------- GEMM (tcgen05)
// C[M x N] = A[M x K] . B[N x K]^T on the fifth-generation tensor cores
// (tcgen05.mma, kind::f16 with BF16 operands, FP32 accumulator in tensor memory).
// One CTA of 256 threads owns a 128 x BN tile of C (BN = 32, so that the small
// GEMMs of the network spread over many SMs):
//  - K advances in chunks of 64, one 128-byte row of BF16 per tile row, through
//    S <= 8 shared-memory stages, all filled at once when K <= 512 (the sizes of
//    this network), so the loads of a tile are in flight together.  Every thread
//    stages its share of a chunk with
//    cp.async in the canonical K-major layout with 128-byte swizzle (8-row groups
//    of 1024 bytes; the 16-byte piece c of row r sits at piece c ^ (r mod 8)),
//    zero-filling rows beyond M or N and columns beyond K.
//  - One thread issues the chunk's MMAs (K = 16 each; the operand descriptors
//    advance 32 bytes per step inside the swizzle atom) and commits them to the
//    stage's mbarrier; a stage is refilled (K > 512) once that barrier has completed.
//  - Epilogue: warp w reads accumulator rows 32 (w mod 4) .. +31 (the tensor-memory
//    lanes its quarter of the SM may access), columns (w / 4) BN/2 .. +BN/2, with
//    tcgen05.ld into the freed stages; the CTA then applies the bias / GELU of
//    `mode` row by row with coalesced stores.
// Every mbarrier wait is bounded; a wait that gives up sets *err, and the CTA
// still frees its tensor memory before it returns.
constexpr int TC_BM = 128, TC_BK = 64, TC_THREADS = 256, TC_BN = 32, TC_MAXS = 8;

__host__ __device__ constexpr uint32_t tc_stage_bytes(int BN) { return (uint32_t)(TC_BM + BN) * 128u; }
// S stages, and room for the epilogue's TC_BM x (BN + 1) float tile and the column
// sums' TC_THREADS partials, plus 1024 bytes of alignment slack
__host__ __device__ constexpr uint32_t tc_smem_bytes(int BN, int S) {
    return ((uint32_t)S * tc_stage_bytes(BN) > ((uint32_t)TC_BM * (BN + 1) + TC_THREADS) * 4u
                ? (uint32_t)S * tc_stage_bytes(BN)
                : ((uint32_t)TC_BM * (BN + 1) + TC_THREADS) * 4u) +
           1024u;
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled
// layout: start address, stride of 1024 bytes between 8-row groups, the sm_100
// descriptor version and the swizzle mode.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;            // leading byte offset (16 B; unused by this layout)
    d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1u << 46;            // version
    d |= (uint64_t)2u << 61;            // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128.
__device__ __forceinline__ uint32_t tc_idesc(int BN) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Tensor memory and stage barriers of a CTA that computes GEMM tiles; the
// barriers' phase parities carry over from tile to tile.
struct TcCtx {
    uint32_t tmem;
    uint64_t* bar;            // TC_MAXS mbarriers in shared memory
    uint32_t ph[TC_MAXS];     // parity of the next phase of each stage's barrier
};
__device__ __forceinline__ void tc_setup(TcCtx& c, uint64_t* bar, uint32_t* tmem_slot, uint32_t ncols) {
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < TC_MAXS; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    c.tmem = *tmem_slot;
    c.bar = bar;
    for (int k = 0; k < TC_MAXS; ++k) c.ph[k] = 0u;
}
__device__ __forceinline__ void tc_teardown(const TcCtx& c, uint32_t ncols) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "r"(ncols) : "memory");
}

// One 128 x BN tile (column tile bx, row tile by, K split bz) of the GEMM g with
// S stages, epilogue included; `base` is the CTA's 1024-byte aligned dynamic
// shared memory.  Operands and the epilogue's inputs are read through L2 only, so
// that tiles see what other CTAs of the same launch wrote before a grid barrier.
// Returns false when a wait for the MMAs gave up.
template <int BN>
__device__ bool gemm_tile(const GemmArgs& g, int S, int bx, int by, int bz, TcCtx& ctx, unsigned char* base) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bm = by * TC_BM, bn = bx * BN;
    const int kbeg = bz * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
    const uint32_t stage = tc_stage_bytes(BN);
    const uint32_t tmem = ctx.tmem;
    uint64_t* bar = ctx.bar;

    auto load = [&](int s, int k0) {
        unsigned char* sa = base + s * stage;
        for (int i = tid; i < (TC_BM + BN) * 8; i += TC_THREADS) {
            const int r = i >> 3, c = i & 7;
            const bool isA = r < TC_BM;
            const int rr = isA ? r : r - TC_BM;
            const int grow = (isA ? bm : bn) + rr, kcol = k0 + c * 8;
            const bool valid = grow < (isA ? g.M : g.N) && kcol < kend;
            const bf16* src = isA ? g.A + (size_t)(valid ? grow : 0) * g.lda + (valid ? kcol : 0)
                                  : g.B + (size_t)(valid ? grow : 0) * g.ldb + (valid ? kcol : 0);
            cp_async16_zfill(sa + r * 128 + ((c ^ (rr & 7)) << 4), src, valid);
        }
        cp_async_commit();
    };

    const int nk = (kend - kbeg + TC_BK - 1) / TC_BK;
    uint32_t* phase = ctx.ph;
    uint32_t pend = 0;  // stages with a commit not yet waited for
    bool ok = true;
    int issued = 0;
    for (; issued < S && issued < nk; ++issued) load(issued, kbeg + issued * TC_BK);
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % S;
        switch (issued - 1 - kt) {  // chunk kt has landed; later chunks may still be in flight
            case 0: cp_async_wait<0>(); break;
            case 1: cp_async_wait<1>(); break;
            case 2: cp_async_wait<2>(); break;
            case 3: cp_async_wait<3>(); break;
            case 4: cp_async_wait<4>(); break;
            case 5: cp_async_wait<5>(); break;
            case 6: cp_async_wait<6>(); break;
            default: cp_async_wait<7>(); break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staged data -> tensor-core reads
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(base + s * stage), b0 = a0 + TC_BM * 128;
            const uint32_t idesc = tc_idesc(BN);
            const int ksteps = min(TC_BK, kend - kbeg - kt * TC_BK) / 16;
            for (int k = 0; k < ksteps; ++k) {
                const uint64_t ad = tc_smem_desc(a0 + 32u * k), bd = tc_smem_desc(b0 + 32u * k);
                const uint32_t acc = (kt > 0 || k > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[s]))
                         : "memory");
        }
        pend |= 1u << s;
        if (kt + S < nk) {  // refill this stage with chunk kt + S once its MMAs have read it
            ok = mbar_wait_bounded(&bar[s], phase[s]) && ok;
            phase[s] ^= 1u;
            pend &= ~(1u << s);
            load(s, kbeg + (kt + S) * TC_BK);
            ++issued;
        }
    }
    // every commit of the tile completes (the last one after every MMA of the tile)
    for (int s = 0; s < S; ++s)
        if ((pend >> s) & 1u) {
            ok = mbar_wait_bounded(&bar[s], phase[s]) && ok;
            phase[s] ^= 1u;
        }
    tc_fence_after();
    // accumulator -> shared memory (the stages are free: every MMA has completed and
    // every copy has landed), then row-wise coalesced stores with the epilogue
    float* tile = reinterpret_cast<float*>(base);  // TC_BM rows of BN + 1 floats
    constexpr int TW = BN + 1;
    const int quarter = warp & 3, half = warp >> 2;
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
        uint32_t v[16];
        const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) tile[(32 * quarter + lane) * TW + c0 + j] = __uint_as_float(v[j]);
    }
    __syncthreads();
    float* const Cz = g.C + (size_t)bz * g.cstride;
    // C (and H) row by row; the tile then holds the value H is made of (0 outside).
    // Eight elements per thread and round: their global operands (bias, Z of the
    // layer below) are loaded together before the arithmetic.
    constexpr int EU = 8;
    for (int i0 = tid; i0 < TC_BM * BN; i0 += TC_THREADS * EU) {
        float xin[EU], aux[EU];
#pragma unroll
        for (int u = 0; u < EU; ++u) {
            const int i = i0 + u * TC_THREADS;
            const int rr = i / BN, cc = i - rr * BN;
            const int r = bm + rr, c = bn + cc;
            const bool in = i < TC_BM * BN && r < g.M && c < g.N;
            const bool valid = in && r < g.Mvalid && c < g.Nvalid;
            xin[u] = i < TC_BM * BN ? tile[rr * TW + cc] : 0.f;
            aux[u] = 0.f;
            if (valid && (g.mode == 1 || g.mode == 2)) aux[u] = __ldcg(&g.bias[c]);
            if (valid && g.mode == 3) aux[u] = __ldcg(&g.Zp[(size_t)r * g.ldz + c]);
        }
#pragma unroll
        for (int u = 0; u < EU; ++u) {
            const int i = i0 + u * TC_THREADS;
            if (i >= TC_BM * BN) continue;
            const int rr = i / BN, cc = i - rr * BN;
            const int r = bm + rr, c = bn + cc;
            float out = 0.f;
            if (r < g.M && c < g.N) {
                const bool valid = r < g.Mvalid && c < g.Nvalid;
                float x = xin[u];
                if (g.mode == 1 || g.mode == 2) x = valid ? x + aux[u] : 0.f;
                if (g.mode == 3) x = valid ? x * gelu_prime_f(aux[u]) : 0.f;
                Cz[(size_t)r * g.ldc + c] = x;
                out = g.mode == 1 ? (valid ? gelu_f(x) : 0.f) : x;
                if (g.mode == 1 || g.mode == 3) g.H[(size_t)r * g.ldh + c] = __float2bfloat16(out);
            }
            tile[rr * TW + cc] = out;
        }
    }
    if (g.HT || g.cs) {
        __syncthreads();
        if (g.HT)  // transposed, coalesced along the rows of C
            for (int i = tid; i < TC_BM * BN; i += TC_THREADS) {
                const int rr = i % TC_BM, cc = i / TC_BM;
                const int r = bm + rr, c = bn + cc;
                if (r < g.M && c < g.N) g.HT[(size_t)c * g.ldht + r] = __float2bfloat16(tile[rr * TW + cc]);
            }
        if (g.cs) {  // fixed order: eight partial sums of 16 rows per column, then their sum
            constexpr int RG = TC_THREADS / BN, RPG = TC_BM / RG;
            float* part = tile + TC_BM * TW;  // RG x BN floats after the tile
            const int c = tid % BN, grp = tid / BN;
            float sum = 0.f;
#pragma unroll 4
            for (int rr = grp * RPG; rr < (grp + 1) * RPG; ++rr) sum += tile[rr * TW + c];
            part[grp * BN + c] = sum;
            __syncthreads();
            if (tid < BN && bn + tid < g.N) {
                float tot = 0.f;
                for (int k = 0; k < RG; ++k) tot += part[k * BN + tid];
                g.cs[(size_t)by * g.ldcs + bn + tid] = tot;
            }
        }
    }
    // the tile's shared memory and accumulator are free again for the CTA's next tile
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return ok;
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) gemm_tc_kernel(const GemmArgs g, int S, int* err) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar[TC_MAXS];
    __shared__ uint32_t tmem_slot;
    constexpr uint32_t ncols = BN <= 32 ? 32u : 64u;
    TcCtx ctx;
    tc_setup(ctx, bar, &tmem_slot, ncols);
    const bool ok = gemm_tile<BN>(g, S, blockIdx.x, blockIdx.y, blockIdx.z, ctx, base);
    if (!ok && (threadIdx.x & 31) == 0) atomicExch(err, 1);
    tc_teardown(ctx, ncols);
}

// ---------------------------------------------------------------- helpers
// BF16 copies of a weight matrix (rows x cols) and of its transpose
__global__ void weights_to_bf16_kernel(const float* W, bf16* Wb, bf16* WbT, int rows, int cols) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)rows * cols; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const bf16 v = __float2bfloat16(W[i]);
        Wb[i] = v;
        WbT[(size_t)c * rows + r] = v;
    }
}

// standardized inputs into the padded bf16 H_0 (rows >= n and columns >= n_in are zero)
// row r of the batch is sample idx[r0 + r] (r0 + r when idx is NULL)
__device__ __forceinline__ size_t sample_row(const int* idx, int64_t r0, int r) {
    return idx ? (size_t)idx[r0 + r] : (size_t)(r0 + r);
}

__device__ __forceinline__ void load_inputs_dev(const float* X, const int* idx, int64_t r0, int n, int n_in,
                                                const float* mu, const float* sd, bf16* H0, int ld, int Bp, bf16* H0T,
                                                size_t first, size_t step) {
    for (size_t i = first; i < (size_t)Bp * ld; i += step) {
        const int r = (int)(i / ld), c = (int)(i % ld);
        float v = 0.f;
        if (r < n && c < n_in) v = (X[sample_row(idx, r0, r) * n_in + c] - mu[c]) / sd[c];
        H0[i] = __float2bfloat16(v);
        if (H0T) H0T[(size_t)c * Bp + r] = __float2bfloat16(v);  // the transpose for the weight gradient
    }
}
__global__ void load_inputs_kernel(const float* X, const int* idx, int64_t r0, int n, int n_in, const float* mu,
                                   const float* sd, bf16* H0, int ld, int Bp, bf16* H0T) {
    load_inputs_dev(X, idx, r0, n, n_in, mu, sd, H0, ld, Bp, H0T, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                    (size_t)gridDim.x * blockDim.x);
}

// dY = 2 (Y - T_std) / (n n_out) into fp32, bf16 and transposed bf16 (padding zero),
// the loss sum, and per LG_ROWS-row tile the column sums of dY in a fixed order (the
// output bias gradient; cs[blockIdx.x * ld + c]).  One block per LG_ROWS x 64 tile
// (grid: row tiles x column tiles), coalesced along the columns; the transposed
// copy and the column sums go through a shared-memory tile.
constexpr int LG_ROWS = 32;
struct LossArgs {
    const float* Y;
    int ldy;
    const float* T;
    const int* idx;
    int64_t r0;
    int n, n_out;
    const float *mu, *sd;
    float* dZ;
    bf16 *dZb, *dZbT;
    int ld, Bp;
    float* cs;
    double* loss;
};
// The LG_ROWS x 64 tile (row tile bx, column tile by); `tile` is LG_ROWS x 65
// floats of shared memory.  Y is read through L2 (written earlier in the same
// launch by the fused epoch).
__device__ void loss_grad_tile(const LossArgs& a, int bx, int by, float (*tile)[65]) {
    const float* Y = a.Y;
    const int ldy = a.ldy, n = a.n, n_out = a.n_out, ld = a.ld, Bp = a.Bp;
    const float* T = a.T;
    const int* idx = a.idx;
    const int64_t r0 = a.r0;
    const float *mu = a.mu, *sd = a.sd;
    float* dZ = a.dZ;
    bf16 *dZb = a.dZb, *dZbT = a.dZbT;
    double s = 0.0;
    const float scale = 2.0f / ((float)n * (float)n_out);
    const int rbeg = bx * LG_ROWS, cbeg = by * 64;
    constexpr int EU = 8;  // elements per thread and round, their loads issued together
    for (int i0 = threadIdx.x; i0 < LG_ROWS * 64; i0 += blockDim.x * EU) {
        float yv[EU], tv[EU];
#pragma unroll
        for (int u = 0; u < EU; ++u) {
            const int i = i0 + u * blockDim.x, rr = i >> 6, cc = i & 63, r = rbeg + rr, c = cbeg + cc;
            const bool in = i < LG_ROWS * 64 && r < n && c < n_out;
            yv[u] = in ? __ldcg(&Y[(size_t)r * ldy + c]) : 0.f;
            tv[u] = in ? __ldg(&T[sample_row(idx, r0, r) * n_out + c]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < EU; ++u) {
            const int i = i0 + u * blockDim.x, rr = i >> 6, cc = i & 63, r = rbeg + rr, c = cbeg + cc;
            if (i >= LG_ROWS * 64) continue;
            float g = 0.f;
            if (r < Bp && c < ld) {
                if (r < n && c < n_out) {
                    const float d = yv[u] - (tv[u] - mu[c]) / sd[c];
                    s += (double)d * d;
                    g = scale * d;
                }
                dZ[(size_t)r * ld + c] = g;
                dZb[(size_t)r * ld + c] = __float2bfloat16(g);
            }
            tile[rr][cc] = g;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < LG_ROWS * 64; i += blockDim.x) {
        const int rr = i % LG_ROWS, cc = i / LG_ROWS, r = rbeg + rr, c = cbeg + cc;
        if (r < Bp && c < ld) dZbT[(size_t)c * Bp + r] = __float2bfloat16(tile[rr][cc]);
    }
    {  // column sums in a fixed order: four partials of LG_ROWS/4 rows per column, then their sum
        __shared__ float part[4][64];
        const int c = threadIdx.x & 63, grp = threadIdx.x >> 6;
        float csum = 0.f;
        if (grp < 4)
            for (int rr = grp * (LG_ROWS / 4); rr < (grp + 1) * (LG_ROWS / 4); ++rr) csum += tile[rr][c];
        if (grp < 4) part[grp][c] = csum;
        __syncthreads();
        if (threadIdx.x < 64 && cbeg + threadIdx.x < ld)
            a.cs[(size_t)bx * ld + cbeg + threadIdx.x] = ((part[0][threadIdx.x] + part[1][threadIdx.x]) +
                                                          part[2][threadIdx.x]) + part[3][threadIdx.x];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(a.loss, s);
    __syncthreads();  // the tile is free for the CTA's next one
}
__global__ void __launch_bounds__(256) loss_grad_kernel(const LossArgs a) {
    __shared__ float tile[LG_ROWS][65];
    loss_grad_tile(a, blockIdx.x, blockIdx.y, tile);
}

// weight gradients: the split-K partials summed in order into the first one
__global__ void weight_grad_kernel(float* gW, int ksplit, size_t nw) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (size_t)gridDim.x * blockDim.x) {
        float s = gW[i];
        for (int z = 1; z < ksplit; ++z) s += gW[(size_t)z * nw + i];
        gW[i] = s;
    }
}

// bias gradients: the tile column sums summed in tile order
__global__ void bias_grad_kernel(const float* cs, int ntiles, int cols, float* gb) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int m = 0; m < ntiles; ++m) s += cs[(size_t)m * cols + c];
    gb[c] = s;
}

// Optimizer state on the device: the Adam step count, the schedule position and
// the hyper-parameters of the current call.  An epoch launch reads the step
// count and schedule position at its start, derives each minibatch's from its
// index, and writes them back at its end.
struct TrainDev {
    long long t;      // Adam steps taken by this handle (bias corrections use t + 1)
    long long sched;  // minibatch steps taken in this call (cosine schedule position)
    long long total;  // minibatch steps of this call
    float lr, lr_end, b1, b2, eps, wd;
    int tc_err;  // a tensor-core GEMM or a grid barrier gave up waiting (never expected)
};

// Adam on FP32 master weights for every layer in one launch: weights (L2 decay)
// with their BF16 copy and its transpose refreshed, then biases, whose gradient
// is the sum of the tile column sums in tile order.
constexpr int kMaxLayers = 17;
struct AdamLayer {
    float *W, *gW, *mW, *vW, *b, *mb, *vb;
    const float* cs;
    bf16 *Wb, *WbT;
    int rows, cols, ntiles;
    int ksplit;  // gW holds ksplit partial gradients of rows x cols, summed in order
};
struct AdamArgs {
    AdamLayer l[kMaxLayers];
    int L;
    const TrainDev* td;
};

// Adam step number t0 + 1 at schedule position sched for layers lo .. hi-1,
// elements first, first + step, ... of those layers' parameters.  The gradients
// are read through L2 (written earlier in the same launch by the fused epoch).
__device__ void adam_dev(const AdamArgs& A, long long t0, long long sched, size_t first, size_t step, int lo = 0,
                         int hi = -1) {
    if (hi < 0) hi = A.L;
    const TrainDev* td = A.td;
    const float t = (float)(t0 + 1);
    const float b1 = td->b1, b2 = td->b2, eps = td->eps;
    const float c1 = 1.f - powf(b1, t), c2 = 1.f - powf(b2, t);
    float lr = td->lr;
    if (td->lr_end >= 0.f)
        lr = td->lr_end + 0.5f * (td->lr - td->lr_end) *
                              (1.f + cospif((float)sched / (float)(td->total > 0 ? td->total : 1)));
    size_t total = 0;
    for (int l = lo; l < hi; ++l) total += (size_t)A.l[l].rows * (A.l[l].cols + 1);
    for (size_t i = first; i < total; i += step) {
        size_t k = i;
        int l = lo;
        while (k >= (size_t)A.l[l].rows * (A.l[l].cols + 1)) {
            k -= (size_t)A.l[l].rows * (A.l[l].cols + 1);
            ++l;
        }
        const AdamLayer& Ly = A.l[l];
        const size_t nw = (size_t)Ly.rows * Ly.cols;
        float *w, *m, *v, gi;
        if (k < nw) {
            w = Ly.W + k; m = Ly.mW + k; v = Ly.vW + k;
            gi = 0.f;
            for (int z = 0; z < Ly.ksplit; ++z) gi += __ldcg(&Ly.gW[(size_t)z * nw + k]);
            gi += td->wd * *w;
        } else {
            const int o = (int)(k - nw);
            w = Ly.b + o; m = Ly.mb + o; v = Ly.vb + o;
            gi = 0.f;
            for (int mt = 0; mt < Ly.ntiles; ++mt) gi += __ldcg(&Ly.cs[(size_t)mt * Ly.rows + o]);
        }
        const float mi = b1 * *m + (1.f - b1) * gi;
        const float vi = b2 * *v + (1.f - b2) * gi * gi;
        *m = mi;
        *v = vi;
        const float wn = *w - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        *w = wn;
        if (k < nw) {
            const bf16 hb = __float2bfloat16(wn);
            const int r = (int)(k / Ly.cols), c = (int)(k % Ly.cols);
            Ly.Wb[k] = hb;
            Ly.WbT[(size_t)c * Ly.rows + r] = hb;
        }
    }
}

// W ~ N(0, 1/fan_in) in the valid region (Box-Muller on Philox draws), zero padding
__global__ void init_weights_kernel(float* W, int rows, int cols, int ld, int ldrows, float sd, uint32_t k0,
                                    uint32_t k1, uint32_t stream) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)ldrows * ld; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / ld), c = (int)(i % ld);
        float v = 0.f;
        if (r < rows && c < cols) {
            uint32_t ctr[4] = {(uint32_t)i, stream, 0u, 0u};
            philox4x32_10(ctr, k0, k1);
            const float u1 = ((float)ctr[0] + 0.5f) * 2.3283064365386963e-10f;
            const float u2 = ((float)ctr[1] + 0.5f) * 2.3283064365386963e-10f;
            v = sd * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
        }
        W[i] = v;
    }
}

__global__ void destandardize_kernel(const float* Y, int ldy, int n, int n_out, const float* mu, const float* sd,
                                     float* out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)n * n_out; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / n_out), c = (int)(i % n_out);
        out[i] = Y[(size_t)r * ldy + c] * sd[c] + mu[c];
    }
}

// ---------------------------------------------------------------- fused epoch
// One training epoch in one cooperative launch.  Every CTA (one per SM) walks
// the phases of each minibatch -- standardized inputs, the forward GEMMs layer
// by layer, the loss gradient, the backward GEMMs of each layer (the weight
// gradient and the input gradient together: both read only dZ_l) and Adam --
// taking the phase's work items (GEMM tiles, loss tiles, element ranges) in
// turn, with a grid barrier between phases: 2L + 2 barriers per minibatch (Adam
// runs inside the backward phases, see below).
// Tensor memory and the stage barriers are set up once per CTA.  The minibatch
// loop needs no host round trip: rows, Adam step and schedule position follow
// from the minibatch index, and the step count is written back at the end.
struct GemmPlan {
    GemmArgs g;
    int S, tx, ty, tz;  // stages; tile grid (column tiles, row tiles, K splits)
};
struct EpochArgs {
    GemmPlan fwd[kMaxLayers], dw[kMaxLayers], dz[kMaxLayers];  // dz[l]: dZ_{l-1} from dZ_l (l >= 1)
    AdamArgs adam;
    LossArgs loss;
    int loss_tx, loss_ty;
    const float* X;
    const int* idx;
    int n_in;
    const float *mu_in, *sd_in;
    bf16 *H0, *H0T;
    int ld0, L, Bp, bs, nmb;
    int64_t n;
    TrainDev* td;
    unsigned *bar_count, *bar_gen;  // grid barrier
    int* abort_flag;                // a barrier wait gave up: every CTA leaves
};

// Grid barrier of a cooperative launch (all CTAs resident): arrive on a counter,
// the last arrival resets it and advances the generation the others wait for.
// Each wait is bounded (about 2 s of SM clock); one that gives up raises the
// abort flag, which every CTA sees at its next barrier.  Returns false on abort.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ bool grid_barrier(unsigned* count, unsigned* gen, int* abort_flag) {
    __shared__ int s_go;
    __syncthreads();  // the CTA's writes before the barrier are ordered before thread 0's release
    if (threadIdx.x == 0) {
        volatile int* vabort = abort_flag;
        const unsigned g0 = ld_acquire_gpu(gen);
        int go = 1;
        unsigned old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
        if (old == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(count) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gen) : "memory");
        } else {
            const long long t0 = clock64();
            while (ld_acquire_gpu(gen) == g0) {
                if (*vabort || clock64() - t0 > 4000000000LL) {
                    atomicExch(abort_flag, 1);
                    go = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (*vabort) go = 0;
        s_go = go;
    }
    __syncthreads();  // every thread's later reads are ordered after thread 0's acquire
    return s_go != 0;
}

__global__ void __launch_bounds__(TC_THREADS, 1) train_epoch_kernel(const __grid_constant__ EpochArgs E) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar[TC_MAXS];
    __shared__ uint32_t tmem_slot;
    TcCtx ctx;
    tc_setup(ctx, bar, &tmem_slot, 32u);
    const long long t0 = E.td->t, s0 = E.td->sched;
    const size_t first = (size_t)blockIdx.x * TC_THREADS + threadIdx.x, step = (size_t)gridDim.x * TC_THREADS;
    bool ok = true, go = true;
    // the tiles of one or two GEMMs as one work list
    auto run = [&](const GemmPlan& p, int mv, const GemmPlan* q, int mvq) {
        const int np = p.tx * p.ty * p.tz, nq = q ? q->tx * q->ty * q->tz : 0;
        for (int t = blockIdx.x; t < np + nq; t += gridDim.x) {
            const GemmPlan& pl = t < np ? p : *q;
            const int u = t < np ? t : t - np;
            GemmArgs g = pl.g;
            const int mvalid = t < np ? mv : mvq;
            if (mvalid >= 0) g.Mvalid = mvalid;
            const int bx = u % pl.tx, rest = u / pl.tx;
            ok = gemm_tile<TC_BN>(g, pl.S, bx, rest % pl.ty, rest / pl.ty, ctx, base) && ok;
        }
    };
    // Adam of layer l runs in the backward phase of layer l-1 (which reads neither
    // W_l nor its gradients' producers), Adam of layer 0 in the next minibatch's
    // input phase (the first forward GEMM reads W_0 after that barrier) or in a
    // last phase of its own
    for (int mb = 0; mb < E.nmb && go; ++mb) {
        const int64_t r0 = (int64_t)mb * E.bs;
        const int nb = (int)min((int64_t)E.bs, E.n - r0);
        load_inputs_dev(E.X, E.idx, r0, nb, E.n_in, E.mu_in, E.sd_in, E.H0, E.ld0, E.Bp, E.H0T, first, step);
        if (mb > 0) adam_dev(E.adam, t0 + mb - 1, s0 + mb - 1, first, step, 0, 1);
        go = grid_barrier(E.bar_count, E.bar_gen, E.abort_flag);
        for (int l = 0; l < E.L && go; ++l) {
            run(E.fwd[l], nb, nullptr, -1);
            go = grid_barrier(E.bar_count, E.bar_gen, E.abort_flag);
        }
        if (!go) break;
        LossArgs la = E.loss;
        la.r0 = r0;
        la.n = nb;
        for (int t = blockIdx.x; t < E.loss_tx * E.loss_ty; t += gridDim.x)
            loss_grad_tile(la, t % E.loss_tx, t / E.loss_tx, reinterpret_cast<float(*)[65]>(base));
        go = grid_barrier(E.bar_count, E.bar_gen, E.abort_flag);
        for (int l = E.L - 1; l >= 0 && go; --l) {
            run(E.dw[l], -1, l > 0 ? &E.dz[l] : nullptr, nb);
            if (l + 1 < E.L) adam_dev(E.adam, t0 + mb, s0 + mb, first, step, l + 1, l + 2);
            go = grid_barrier(E.bar_count, E.bar_gen, E.abort_flag);
        }
    }
    if (go && E.nmb > 0) {
        adam_dev(E.adam, t0 + E.nmb - 1, s0 + E.nmb - 1, first, step, 0, 1);
        go = grid_barrier(E.bar_count, E.bar_gen, E.abort_flag);
    }
    if (go && blockIdx.x == 0 && threadIdx.x == 0) {
        E.td->t = t0 + E.nmb;
        E.td->sched = s0 + E.nmb;
    }
    if ((!ok || !go) && threadIdx.x == 0) atomicExch(&E.td->tc_err, 1);
    tc_teardown(ctx, 32u);
}

}  // namespace cl

// ---------------------------------------------------------------- host side

struct cl_surrogate {
    int n_in, n_out, width, depth, L;
    std::vector<int> d, P;  // true and padded dims of layer inputs/outputs (size L+1)
    std::vector<float*> W, gW, mW, vW, b, gb, mb, vb;
    std::vector<cl::bf16*> Wb, WbT;
    cudaStream_t stream;
    int Bp = 0;  // batch capacity (padded)
    std::vector<float*> Z;         // per layer: Bp x P[l+1] fp32
    std::vector<cl::bf16*> H;      // per layer input: Bp x P[l] bf16
    std::vector<cl::bf16*> HT;     // transposes: P[l] x Bp (written by the producing kernel)
    std::vector<float*> cs;        // per layer: column sums of dZ_l per 128-row tile (bias gradients)
    float* dZ[2] = {nullptr, nullptr};          // Bp x maxP fp32, alternating between layers
    cl::bf16* dZb[2] = {nullptr, nullptr};      // Bp x maxP
    cl::bf16* dZbT[2] = {nullptr, nullptr};     // maxP x Bp
    float *Xd = nullptr, *Td = nullptr;  // raw data (n x n_in / n x n_out) for the current call
    size_t cap_n = 0;
    float *mu_in, *sd_in, *mu_out, *sd_out;  // standardization (device, length n_in / n_out)
    std::vector<float> h_mu_in, h_sd_in, h_mu_out, h_sd_out;
    double* dloss = nullptr;
    cl::TrainDev* tdev = nullptr;  // device optimizer state
    int* d_perm = nullptr;         // sample order of the current epoch
    int64_t perm_cap = 0;
    long long gen = 0;  // counts reallocations of the buffers
    long long epochs_done = 0;
    uint64_t seed = 0;
    int sms = 1;
    std::vector<cl::GemmPlan>* record = nullptr;  // set: gemm() records its plan instead of launching
    unsigned* d_gridbar = nullptr;                // fused epoch: barrier counter, generation, abort flag
};

namespace {

inline int pad32(int x) { return (x + 31) / 32 * 32; }

cl_status sfail(cl_status s, const std::string& m) {
    cl::set_global_error(m.c_str());
    return s;
}

// Optional fused outputs of a GEMM: the pre-activations of mode 3, the
// transposed bf16 output, the per-tile column sums.
struct GemmExtra {
    const float* Zp = nullptr;
    int ldz = 0;
    cl::bf16* HT = nullptr;
    int ldht = 0;
    float* cs = nullptr;
    int ldcs = 0;
    int kchunk = 0;  // > 0: split K into chunks of this size, partial C matrices one after the other
};

// Split-K of the weight-gradient GEMMs (K = the batch): up to 4 splits of at least
// 128 rows, so that more CTAs share the longest K loops.
constexpr int kMaxSplits = 4;
inline int dw_kchunk(int Bp) {
    const int want = std::min(kMaxSplits, (Bp + 127) / 128);
    return (Bp + want * cl::TC_BK - 1) / (want * cl::TC_BK) * cl::TC_BK;
}
inline int dw_splits(int Bp) { return (Bp + dw_kchunk(Bp) - 1) / dw_kchunk(Bp); }

void gemm(cl_surrogate* S, const cl::bf16* A, int lda, const cl::bf16* B, int ldb, float* C, int ldc, int M, int N,
          int K, int mode, const float* bias, cl::bf16* H, int ldh, int Mvalid, int Nvalid,
          const GemmExtra& x = GemmExtra()) {
    cl::GemmArgs g;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc; g.M = M; g.N = N; g.K = K;
    g.mode = mode; g.bias = bias; g.H = H; g.ldh = ldh; g.Mvalid = Mvalid; g.Nvalid = Nvalid;
    g.Zp = x.Zp; g.ldz = x.ldz; g.HT = x.HT; g.ldht = x.ldht; g.cs = x.cs; g.ldcs = x.ldcs;
    g.kchunk = x.kchunk > 0 ? x.kchunk : K;
    g.cstride = (size_t)M * ldc;
    const int splits = (K + g.kchunk - 1) / g.kchunk;
    constexpr int BN = cl::TC_BN;  // N is a multiple of 32
    const int nk = (g.kchunk + cl::TC_BK - 1) / cl::TC_BK;
    const int stages = nk < cl::TC_MAXS ? nk : cl::TC_MAXS;
    if (S->record) {
        cl::GemmPlan p;
        p.g = g;
        p.S = stages;
        p.tx = (N + BN - 1) / BN;
        p.ty = (M + cl::TC_BM - 1) / cl::TC_BM;
        p.tz = splits;
        S->record->push_back(p);
        return;
    }
    static bool attr_set = false;  // the stage ring needs the opt-in shared-memory size
    if (!attr_set) {
        cudaFuncSetAttribute(cl::gemm_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cl::tc_smem_bytes(BN, cl::TC_MAXS));
        // one shared-memory carveout for the per-launch kernels, so that consecutive
        // launches need no reconfiguration of the SMs' L1/shared split
        const void* fns[] = {(const void*)cl::gemm_tc_kernel<BN>, (const void*)cl::loss_grad_kernel,
                             (const void*)cl::load_inputs_kernel};
        for (const void* f : fns) cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaGetLastError();
        attr_set = true;
    }
    dim3 grid((N + BN - 1) / BN, (M + cl::TC_BM - 1) / cl::TC_BM, splits);
    cl::gemm_tc_kernel<BN><<<grid, cl::TC_THREADS, cl::tc_smem_bytes(BN, stages), S->stream>>>(g, stages,
                                                                                                 &S->tdev->tc_err);
}

// CL_ERR_TIMEOUT when a tensor-core GEMM of the last call gave up waiting (after a synchronize)
cl_status check_tc(cl_surrogate* S, const char* who) {
    int flag = 0;
    if (cudaMemcpy(&flag, &S->tdev->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return sfail(CL_ERR_CUDA, std::string(who) + ": reading the GEMM status");
    if (flag) return sfail(CL_ERR_TIMEOUT, std::string(who) + ": a tensor-core GEMM timed out waiting for its MMAs");
    return CL_OK;
}

// row tiles of the bias gradient's column sums of layer l: the output layer's come
// from the loss gradient (LG_ROWS rows each), the others from the GEMM epilogue
// that produces dZ_l (TC_BM rows each)
int bias_tiles(const cl_surrogate* S, int l, int Bp) {
    const int rows = l == S->L - 1 ? cl::LG_ROWS : cl::TC_BM;
    return (Bp + rows - 1) / rows;
}

cl_status ensure_batch(cl_surrogate* S, int n) {
    const int Bp = (n + 63) / 64 * 64;
    if (Bp <= S->Bp) return CL_OK;
    for (auto p : S->Z) cudaFree(p);
    for (auto p : S->H) cudaFree(p);
    for (auto p : S->HT) cudaFree(p);
    for (auto p : S->cs) cudaFree(p);
    for (int k = 0; k < 2; ++k) { cudaFree(S->dZ[k]); cudaFree(S->dZb[k]); cudaFree(S->dZbT[k]); }
    S->Z.assign(S->L, nullptr);
    S->H.assign(S->L, nullptr);
    S->HT.assign(S->L, nullptr);
    S->cs.assign(S->L, nullptr);
    int maxP = 0;
    for (int p : S->P) maxP = std::max(maxP, p);
    bool ok = true;
    for (int l = 0; l < S->L; ++l) {
        const int ntiles = bias_tiles(S, l, Bp);
        ok = ok && cudaMalloc(&S->Z[l], sizeof(float) * Bp * S->P[l + 1]) == cudaSuccess;
        ok = ok && cudaMalloc(&S->H[l], sizeof(cl::bf16) * Bp * S->P[l]) == cudaSuccess;
        ok = ok && cudaMalloc(&S->HT[l], sizeof(cl::bf16) * Bp * S->P[l]) == cudaSuccess;
        ok = ok && cudaMalloc(&S->cs[l], sizeof(float) * ntiles * S->P[l + 1]) == cudaSuccess;
    }
    for (int k = 0; k < 2; ++k) {
        ok = ok && cudaMalloc(&S->dZ[k], sizeof(float) * Bp * maxP) == cudaSuccess;
        ok = ok && cudaMalloc(&S->dZb[k], sizeof(cl::bf16) * Bp * maxP) == cudaSuccess;
        ok = ok && cudaMalloc(&S->dZbT[k], sizeof(cl::bf16) * Bp * maxP) == cudaSuccess;
    }
    if (!ok) return sfail(CL_ERR_OOM, "surrogate: activation buffers");
    S->Bp = Bp;
    ++S->gen;
    return CL_OK;
}

cl_status ensure_data(cl_surrogate* S, size_t n) {
    if (n <= S->cap_n) return CL_OK;
    cudaFree(S->Xd);
    cudaFree(S->Td);
    if (cudaMalloc(&S->Xd, sizeof(float) * n * S->n_in) != cudaSuccess ||
        cudaMalloc(&S->Td, sizeof(float) * n * S->n_out) != cudaSuccess)
        return sfail(CL_ERR_OOM, "surrogate: data buffers");
    S->cap_n = n;
    ++S->gen;
    return CL_OK;
}

void refresh_bf16(cl_surrogate* S) {
    for (int l = 0; l < S->L; ++l)
        cl::weights_to_bf16_kernel<<<S->sms * 4, 256, 0, S->stream>>>(S->W[l], S->Wb[l], S->WbT[l], S->P[l + 1],
                                                                       S->P[l]);
}

// forward over batch rows r = 0..n-1, sample idx[r0 + r] (r0 + r without idx) of
// the data in S->Xd, standardized by mu/sd; `training` also writes the transposed
// activations that the weight gradients read
void forward(cl_surrogate* S, const int* idx, int64_t r0, int n, bool training) {
    if (!S->record)
        cl::load_inputs_kernel<<<S->sms * 4, 256, 0, S->stream>>>(S->Xd, idx, r0, n, S->n_in, S->mu_in, S->sd_in,
                                                                  S->H[0], S->P[0], S->Bp, training ? S->HT[0] : nullptr);
    for (int l = 0; l < S->L; ++l) {
        const bool last = l == S->L - 1;
        GemmExtra x;
        if (training && !last) {
            x.HT = S->HT[l + 1];
            x.ldht = S->Bp;
        }
        gemm(S, S->H[l], S->P[l], S->Wb[l], S->P[l], S->Z[l], S->P[l + 1], S->Bp, S->P[l + 1], S->P[l], last ? 2 : 1,
             S->b[l], last ? nullptr : S->H[l + 1], S->P[l + 1], n, S->d[l + 1], x);
    }
}

cl::LossArgs loss_args(cl_surrogate* S, const int* idx, int64_t r0, int n, int cur) {
    const int L = S->L;
    cl::LossArgs a;
    a.Y = S->Z[L - 1]; a.ldy = S->P[L]; a.T = S->Td; a.idx = idx; a.r0 = r0; a.n = n; a.n_out = S->n_out;
    a.mu = S->mu_out; a.sd = S->sd_out; a.dZ = S->dZ[cur]; a.dZb = S->dZb[cur]; a.dZbT = S->dZbT[cur];
    a.ld = S->P[L]; a.Bp = S->Bp; a.cs = S->cs[L - 1]; a.loss = S->dloss;
    return a;
}

// backward: weight gradients into gW, the bias gradients as tile column sums in
// cs (summed by the optimizer, or by bias_grads); loss sum added into S->dloss.
// Per layer two GEMMs: dW_l = dZ_l^T H_l, and dZ_{l-1} = (dZ_l W_l) GELU'(Z_{l-1})
// with the elementwise factor, the transposed copy and the column sums fused
// into its epilogue.
void backward(cl_surrogate* S, const int* idx, int64_t r0, int n) {
    const int L = S->L, Bp = S->Bp;
    int cur = 0;
    if (!S->record)
        cl::loss_grad_kernel<<<dim3((Bp + cl::LG_ROWS - 1) / cl::LG_ROWS, (S->P[L] + 63) / 64), 256, 0,
                               S->stream>>>(loss_args(S, idx, r0, n, cur));
    for (int l = L - 1; l >= 0; --l) {
        const int Pin = S->P[l], Pout = S->P[l + 1];
        GemmExtra xw;
        xw.kchunk = dw_kchunk(Bp);  // partial gradients, summed by the optimizer
        gemm(S, S->dZbT[cur], Bp, S->HT[l], Bp, S->gW[l], Pin, Pout, Pin, Bp, 0, nullptr, nullptr, 0, Pout, Pin, xw);
        if (l > 0) {
            GemmExtra x;
            x.Zp = S->Z[l - 1];
            x.ldz = Pin;
            x.HT = S->dZbT[1 - cur];
            x.ldht = Bp;
            x.cs = S->cs[l - 1];
            x.ldcs = Pin;
            gemm(S, S->dZb[cur], Pout, S->WbT[l], Pout, S->dZ[1 - cur], Pin, Bp, Pin, Pout, 3, nullptr, S->dZb[1 - cur],
                 Pin, n, S->d[l], x);
            cur = 1 - cur;
        }
    }
}

cl::AdamArgs adam_args(cl_surrogate* S) {
    cl::AdamArgs a;
    memset(&a, 0, sizeof(a));
    a.L = S->L;
    a.td = S->tdev;
    for (int l = 0; l < S->L; ++l) {
        cl::AdamLayer& y = a.l[l];
        y.W = S->W[l]; y.gW = S->gW[l]; y.mW = S->mW[l]; y.vW = S->vW[l];
        y.b = S->b[l]; y.mb = S->mb[l]; y.vb = S->vb[l];
        y.cs = S->cs[l];
        y.Wb = S->Wb[l]; y.WbT = S->WbT[l];
        y.rows = S->P[l + 1];
        y.cols = S->P[l];
        y.ntiles = bias_tiles(S, l, S->Bp);
        y.ksplit = dw_splits(S->Bp);
    }
    return a;
}

// bias gradients gb from the tile column sums and the weight gradients from the
// split partials (for the gradient query)
void bias_grads(cl_surrogate* S) {
    for (int l = 0; l < S->L; ++l)
        cl::weight_grad_kernel<<<S->sms * 2, 256, 0, S->stream>>>(S->gW[l], dw_splits(S->Bp),
                                                                  (size_t)S->P[l + 1] * S->P[l]);
    for (int l = 0; l < S->L; ++l)
        cl::bias_grad_kernel<<<(S->P[l + 1] + 127) / 128, 128, 0, S->stream>>>(S->cs[l], bias_tiles(S, l, S->Bp),
                                                                               S->P[l + 1], S->gb[l]);
}

void set_identity_scaling(cl_surrogate* S) {
    S->h_mu_in.assign(S->n_in, 0.f);
    S->h_sd_in.assign(S->n_in, 1.f);
    S->h_mu_out.assign(S->n_out, 0.f);
    S->h_sd_out.assign(S->n_out, 1.f);
}

void upload_scaling(cl_surrogate* S) {
    cudaMemcpyAsync(S->mu_in, S->h_mu_in.data(), sizeof(float) * S->n_in, cudaMemcpyHostToDevice, S->stream);
    cudaMemcpyAsync(S->sd_in, S->h_sd_in.data(), sizeof(float) * S->n_in, cudaMemcpyHostToDevice, S->stream);
    cudaMemcpyAsync(S->mu_out, S->h_mu_out.data(), sizeof(float) * S->n_out, cudaMemcpyHostToDevice, S->stream);
    cudaMemcpyAsync(S->sd_out, S->h_sd_out.data(), sizeof(float) * S->n_out, cudaMemcpyHostToDevice, S->stream);
}

}  // namespace

extern "C" {

cl_status surrogate_destroy(cl_surrogate* S) {
    if (!S) return CL_OK;
    for (auto* v : {&S->W, &S->gW, &S->mW, &S->vW, &S->b, &S->gb, &S->mb, &S->vb})
        for (auto p : *v) cudaFree(p);
    for (auto p : S->Wb) cudaFree(p);
    for (auto p : S->WbT) cudaFree(p);
    for (auto p : S->Z) cudaFree(p);
    for (auto p : S->H) cudaFree(p);
    for (auto p : S->HT) cudaFree(p);
    for (auto p : S->cs) cudaFree(p);
    for (int k = 0; k < 2; ++k) { cudaFree(S->dZ[k]); cudaFree(S->dZb[k]); cudaFree(S->dZbT[k]); }
    cudaFree(S->Xd); cudaFree(S->Td);
    cudaFree(S->mu_in); cudaFree(S->sd_in); cudaFree(S->mu_out); cudaFree(S->sd_out);
    cudaFree(S->dloss);
    cudaFree(S->tdev);
    cudaFree(S->d_perm);
    cudaFree(S->d_gridbar);
    delete S;
    return CL_OK;
}

cl_status surrogate_create(int32_t n_in, int32_t n_out, int32_t width, int32_t depth, uint64_t seed, void* stream,
                           cl_surrogate** out) {
    if (!out) return sfail(CL_ERR_ARG, "surrogate_create: out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_in > 1024 || n_out < 1 || n_out > 1024 || width < 1 || width > 4096 || depth < 1 || depth > 16)
        return sfail(CL_ERR_ARG, "surrogate_create: n_in, n_out in [1, 1024], width in [1, 4096], depth in [1, 16]");
    cl_surrogate* S = new cl_surrogate();
    S->n_in = n_in; S->n_out = n_out; S->width = width; S->depth = depth; S->L = depth + 1;
    S->stream = (cudaStream_t)stream;
    S->seed = seed;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, dev);
    S->d.push_back(n_in);
    for (int i = 0; i < depth; ++i) S->d.push_back(width);
    S->d.push_back(n_out);
    for (int x : S->d) S->P.push_back(pad32(x));
    bool ok = true;
    for (int l = 0; l < S->L; ++l) {
        const size_t nw = (size_t)S->P[l + 1] * S->P[l], nb = S->P[l + 1];
        float *w = nullptr, *gw = nullptr, *mw = nullptr, *vw = nullptr, *bb = nullptr, *gbb = nullptr,
              *mbb = nullptr, *vbb = nullptr;
        cl::bf16 *wb = nullptr, *wbt = nullptr;
        ok = ok && cudaMalloc(&w, nw * 4) == cudaSuccess && cudaMalloc(&gw, nw * 4 * kMaxSplits) == cudaSuccess &&
             cudaMalloc(&mw, nw * 4) == cudaSuccess && cudaMalloc(&vw, nw * 4) == cudaSuccess &&
             cudaMalloc(&bb, nb * 4) == cudaSuccess && cudaMalloc(&gbb, nb * 4) == cudaSuccess &&
             cudaMalloc(&mbb, nb * 4) == cudaSuccess && cudaMalloc(&vbb, nb * 4) == cudaSuccess &&
             cudaMalloc(&wb, nw * 2) == cudaSuccess && cudaMalloc(&wbt, nw * 2) == cudaSuccess;
        if (!ok) {
            // this layer's buffers are not yet owned by S: release the ones that were allocated
            for (void* p : {(void*)w, (void*)gw, (void*)mw, (void*)vw, (void*)bb, (void*)gbb, (void*)mbb, (void*)vbb,
                            (void*)wb, (void*)wbt})
                cudaFree(p);
            break;
        }
        S->W.push_back(w); S->gW.push_back(gw); S->mW.push_back(mw); S->vW.push_back(vw);
        S->b.push_back(bb); S->gb.push_back(gbb); S->mb.push_back(mbb); S->vb.push_back(vbb);
        S->Wb.push_back(wb); S->WbT.push_back(wbt);
        cudaMemsetAsync(gw, 0, nw * 4 * kMaxSplits, S->stream); cudaMemsetAsync(mw, 0, nw * 4, S->stream);
        cudaMemsetAsync(vw, 0, nw * 4, S->stream); cudaMemsetAsync(bb, 0, nb * 4, S->stream);
        cudaMemsetAsync(gbb, 0, nb * 4, S->stream); cudaMemsetAsync(mbb, 0, nb * 4, S->stream);
        cudaMemsetAsync(vbb, 0, nb * 4, S->stream);
        cl::init_weights_kernel<<<S->sms * 4, 256, 0, S->stream>>>(w, S->d[l + 1], S->d[l], S->P[l], S->P[l + 1],
                                                                   1.0f / sqrtf((float)S->d[l]),
                                                                   (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                                   (uint32_t)l);
    }
    ok = ok && cudaMalloc(&S->mu_in, 4 * n_in) == cudaSuccess && cudaMalloc(&S->sd_in, 4 * n_in) == cudaSuccess &&
         cudaMalloc(&S->mu_out, 4 * n_out) == cudaSuccess && cudaMalloc(&S->sd_out, 4 * n_out) == cudaSuccess &&
         cudaMalloc(&S->dloss, sizeof(double)) == cudaSuccess && cudaMalloc(&S->tdev, sizeof(cl::TrainDev)) == cudaSuccess &&
         cudaMalloc(&S->d_gridbar, 4 * sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        surrogate_destroy(S);
        return sfail(CL_ERR_OOM, "surrogate_create: parameters");
    }
    set_identity_scaling(S);
    upload_scaling(S);
    refresh_bf16(S);
    cudaMemsetAsync(S->tdev, 0, sizeof(cl::TrainDev), S->stream);
    if (cudaStreamSynchronize(S->stream) != cudaSuccess) {
        surrogate_destroy(S);
        return sfail(CL_ERR_CUDA, "surrogate_create: initialisation");
    }
    *out = S;
    return CL_OK;
}

int64_t surrogate_param_count(const cl_surrogate* S) {
    if (!S) return 0;
    int64_t n = 0;
    for (int l = 0; l < S->L; ++l) n += (int64_t)S->d[l + 1] * S->d[l] + S->d[l + 1];
    return n;
}

// theta: W_0 (d1 x d0 row-major), b_0, W_1, b_1, ... in double
static cl_status copy_params(cl_surrogate* S, double* out, const double* in, bool grads) {
    std::vector<float> buf;
    size_t o = 0;
    for (int l = 0; l < S->L; ++l) {
        const int r = S->d[l + 1], c = S->d[l], ld = S->P[l];
        float* Wd = grads ? S->gW[l] : S->W[l];
        float* bd = grads ? S->gb[l] : S->b[l];
        buf.resize((size_t)r * c);
        if (in) {
            for (size_t i = 0; i < buf.size(); ++i) buf[i] = (float)in[o + i];
            cudaMemcpy2DAsync(Wd, ld * 4, buf.data(), c * 4, c * 4, r, cudaMemcpyHostToDevice, S->stream);
            cudaStreamSynchronize(S->stream);
        } else {
            cudaMemcpy2DAsync(buf.data(), c * 4, Wd, ld * 4, c * 4, r, cudaMemcpyDeviceToHost, S->stream);
            cudaStreamSynchronize(S->stream);
            for (size_t i = 0; i < buf.size(); ++i) out[o + i] = buf[i];
        }
        o += buf.size();
        buf.resize(r);
        if (in) {
            for (int i = 0; i < r; ++i) buf[i] = (float)in[o + i];
            cudaMemcpyAsync(bd, buf.data(), r * 4, cudaMemcpyHostToDevice, S->stream);
            cudaStreamSynchronize(S->stream);
        } else {
            cudaMemcpyAsync(buf.data(), bd, r * 4, cudaMemcpyDeviceToHost, S->stream);
            cudaStreamSynchronize(S->stream);
            for (int i = 0; i < r; ++i) out[o + i] = buf[i];
        }
        o += r;
    }
    if (in) refresh_bf16(S);
    cudaError_t e = cudaStreamSynchronize(S->stream);
    return e == cudaSuccess ? CL_OK : sfail(CL_ERR_CUDA, "surrogate: parameter copy");
}

cl_status surrogate_get_params(cl_surrogate* S, double* theta) {
    if (!S || !theta) return sfail(CL_ERR_ARG, "surrogate_get_params: NULL argument");
    return copy_params(S, theta, nullptr, false);
}

cl_status surrogate_set_params(cl_surrogate* S, const double* theta) {
    if (!S || !theta) return sfail(CL_ERR_ARG, "surrogate_set_params: NULL argument");
    return copy_params(S, nullptr, theta, false);
}

cl_status surrogate_loss_grad(cl_surrogate* S, const float* X, const float* T, int64_t n, double* loss, double* grad) {
    if (!S || !X || !T || n < 1 || n > (1 << 24)) return sfail(CL_ERR_ARG, "surrogate_loss_grad: bad arguments");
    cl_status s = ensure_batch(S, (int)n);
    if (s == CL_OK) s = ensure_data(S, n);
    if (s != CL_OK) return s;
    // raw inputs and targets: identity scaling for this call
    std::vector<float> mi = S->h_mu_in, si = S->h_sd_in, mo = S->h_mu_out, so = S->h_sd_out;
    set_identity_scaling(S);
    upload_scaling(S);
    cudaMemcpyAsync(S->Xd, X, sizeof(float) * n * S->n_in, cudaMemcpyHostToDevice, S->stream);
    cudaMemcpyAsync(S->Td, T, sizeof(float) * n * S->n_out, cudaMemcpyHostToDevice, S->stream);
    cudaMemsetAsync(S->dloss, 0, sizeof(double), S->stream);
    forward(S, nullptr, 0, (int)n, true);
    backward(S, nullptr, 0, (int)n);
    bias_grads(S);
    double l = 0;
    cudaMemcpyAsync(&l, S->dloss, sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    cudaError_t e = cudaStreamSynchronize(S->stream);
    S->h_mu_in = mi; S->h_sd_in = si; S->h_mu_out = mo; S->h_sd_out = so;
    upload_scaling(S);
    if (e != cudaSuccess) return sfail(CL_ERR_CUDA, std::string("surrogate_loss_grad: ") + cudaGetErrorString(e));
    s = check_tc(S, "surrogate_loss_grad");
    if (s != CL_OK) return s;
    if (loss) *loss = l / ((double)n * S->n_out);
    if (grad) return copy_params(S, grad, nullptr, true);
    return CL_OK;
}

// Arguments of the fused epoch for n rows in minibatches of bs (sample order idx)
// on the current buffers: the GEMM plans are the ones forward() and backward()
// would launch for a full minibatch, recorded instead of launched.
cl_status make_epoch(cl_surrogate* S, const int* idx, int64_t n, int bs, cl::EpochArgs& E, size_t& smem) {
    std::vector<cl::GemmPlan> rec;
    S->record = &rec;
    forward(S, idx, 0, bs, true);
    backward(S, idx, 0, bs);
    S->record = nullptr;
    const int L = S->L;
    if ((int)rec.size() != 3 * L - 1) return sfail(CL_ERR_CUDA, "surrogate_train: epoch plan");
    memset(&E, 0, sizeof(E));
    size_t k = 0;
    for (int l = 0; l < L; ++l) E.fwd[l] = rec[k++];
    for (int l = L - 1; l >= 0; --l) {
        E.dw[l] = rec[k++];
        if (l > 0) E.dz[l] = rec[k++];
    }
    E.adam = adam_args(S);
    E.loss = loss_args(S, idx, 0, bs, 0);
    E.loss_tx = (S->Bp + cl::LG_ROWS - 1) / cl::LG_ROWS;
    E.loss_ty = (S->P[L] + 63) / 64;
    E.X = S->Xd;
    E.idx = idx;
    E.n_in = S->n_in;
    E.mu_in = S->mu_in;
    E.sd_in = S->sd_in;
    E.H0 = S->H[0];
    E.H0T = S->HT[0];
    E.ld0 = S->P[0];
    E.L = L;
    E.Bp = S->Bp;
    E.bs = bs;
    E.nmb = (int)((n + bs - 1) / bs);
    E.n = n;
    E.td = S->tdev;
    E.bar_count = S->d_gridbar;
    E.bar_gen = S->d_gridbar + 1;
    E.abort_flag = reinterpret_cast<int*>(S->d_gridbar + 2);
    smem = 1024 + (size_t)cl::LG_ROWS * 65 * sizeof(float);
    for (const auto& p : rec) smem = std::max<size_t>(smem, cl::tc_smem_bytes(cl::TC_BN, p.S));
    return CL_OK;
}

cl_status surrogate_train(cl_surrogate* S, const float* X, const float* Y, int64_t n, const cl_train_cfg* cfg,
                          float* loss_history) {
    if (!S || !X || !Y || !cfg || n < 1 || n > (1 << 24) || cfg->epochs < 1 || cfg->batch < 1 || !(cfg->lr > 0))
        return sfail(CL_ERR_ARG, "surrogate_train: bad arguments");
    const int bs = (int)std::min<int64_t>(cfg->batch, n);
    cl_status s = ensure_batch(S, bs);
    if (s == CL_OK) s = ensure_data(S, n);
    if (s != CL_OK) return s;
    // standardization of inputs and outputs from the training set
    set_identity_scaling(S);
    if (cfg->standardize) {
        for (int c = 0; c < S->n_in; ++c) {
            double m = 0, v = 0;
            for (int64_t i = 0; i < n; ++i) m += X[i * S->n_in + c];
            m /= n;
            for (int64_t i = 0; i < n; ++i) v += (X[i * S->n_in + c] - m) * (X[i * S->n_in + c] - m);
            S->h_mu_in[c] = (float)m;
            S->h_sd_in[c] = (float)std::max(sqrt(v / n), 1e-12);
        }
        for (int c = 0; c < S->n_out; ++c) {
            double m = 0, v = 0;
            for (int64_t i = 0; i < n; ++i) m += Y[i * S->n_out + c];
            m /= n;
            for (int64_t i = 0; i < n; ++i) v += (Y[i * S->n_out + c] - m) * (Y[i * S->n_out + c] - m);
            S->h_mu_out[c] = (float)m;
            S->h_sd_out[c] = (float)std::max(sqrt(v / n), 1e-12);
        }
    }
    upload_scaling(S);
    cudaMemcpyAsync(S->Xd, X, sizeof(float) * n * S->n_in, cudaMemcpyHostToDevice, S->stream);
    cudaMemcpyAsync(S->Td, Y, sizeof(float) * n * S->n_out, cudaMemcpyHostToDevice, S->stream);
    const int64_t per_epoch = (n + bs - 1) / bs;
    cl::TrainDev td;
    // keep the handle's Adam step count, reset the schedule to this call
    if (cudaMemcpyAsync(&td, S->tdev, sizeof(td), cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
        cudaStreamSynchronize(S->stream) != cudaSuccess)
        return sfail(CL_ERR_CUDA, "surrogate_train: optimizer state");
    td.sched = 0;
    td.total = per_epoch * cfg->epochs;
    td.lr = cfg->lr;
    td.lr_end = cfg->lr_end;
    td.b1 = cfg->beta1 > 0 ? cfg->beta1 : 0.9f;
    td.b2 = cfg->beta2 > 0 ? cfg->beta2 : 0.999f;
    td.eps = cfg->eps > 0 ? cfg->eps : 1e-8f;
    td.wd = cfg->weight_decay;
    cudaMemcpyAsync(S->tdev, &td, sizeof(td), cudaMemcpyHostToDevice, S->stream);
    const int shuf = cfg->shuffle ? 1 : 0;
    std::vector<int> perm;
    if (shuf) {
        if (n > S->perm_cap) {
            cudaFree(S->d_perm);
            S->d_perm = nullptr;
            if (cudaMalloc(&S->d_perm, sizeof(int) * n) != cudaSuccess) return sfail(CL_ERR_OOM, "surrogate_train: order");
            S->perm_cap = n;
            ++S->gen;
        }
        perm.resize(n);
    }
    // one epoch = one cooperative launch of the fused epoch kernel (one CTA per SM)
    cl::EpochArgs E;
    size_t smem = 0;
    s = make_epoch(S, shuf ? S->d_perm : nullptr, n, bs, E, smem);
    if (s != CL_OK) return s;
    {
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(cl::train_epoch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cl::tc_smem_bytes(cl::TC_BN, cl::TC_MAXS));
            attr_set = true;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cl::train_epoch_kernel, cl::TC_THREADS, smem) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            return sfail(CL_ERR_CUDA, "surrogate_train: the fused epoch does not fit on an SM");
        }
    }
    for (int ep = 0; ep < cfg->epochs; ++ep) {
        if (shuf) {
            // Fisher-Yates with a 64-bit LCG (Knuth's MMIX constants) keyed by the
            // handle's seed and its epoch count
            for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
            uint64_t x = S->seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(S->epochs_done + 1));
            for (int64_t i = n - 1; i > 0; --i) {
                x = x * 6364136223846793005ull + 1442695040888963407ull;
                const int64_t j = (int64_t)((x >> 33) % (uint64_t)(i + 1));
                std::swap(perm[i], perm[j]);
            }
            cudaMemcpyAsync(S->d_perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, S->stream);
        }
        cudaMemsetAsync(S->dloss, 0, sizeof(double), S->stream);
        cudaMemsetAsync(S->d_gridbar, 0, 4 * sizeof(unsigned), S->stream);
        void* args[] = {&E};
        cudaError_t le = cudaLaunchCooperativeKernel((const void*)cl::train_epoch_kernel, dim3(S->sms),
                                                     dim3(cl::TC_THREADS), args, smem, S->stream);
        if (le != cudaSuccess)
            return sfail(CL_ERR_CUDA, std::string("surrogate_train: epoch launch: ") + cudaGetErrorString(le));
        ++S->epochs_done;
        if (loss_history || shuf) {
            // the host order buffer is rewritten next epoch: wait for this one
            double l = 0;
            if (loss_history) cudaMemcpyAsync(&l, S->dloss, sizeof(double), cudaMemcpyDeviceToHost, S->stream);
            if (cudaStreamSynchronize(S->stream) != cudaSuccess) return sfail(CL_ERR_CUDA, "surrogate_train");
            if (loss_history) loss_history[ep] = (float)(l / ((double)n * S->n_out));
        }
    }
    cudaError_t e = cudaStreamSynchronize(S->stream);
    return e == cudaSuccess ? check_tc(S, "surrogate_train")
                            : sfail(CL_ERR_CUDA, std::string("surrogate_train: ") + cudaGetErrorString(e));
}

cl_status surrogate_predict(cl_surrogate* S, const float* X, int64_t n, float* Y) {
    if (!S || !X || !Y || n < 1 || n > (1 << 24)) return sfail(CL_ERR_ARG, "surrogate_predict: bad arguments");
    cl_status s = ensure_batch(S, (int)std::min<int64_t>(n, 8192));
    if (s == CL_OK) s = ensure_data(S, n);
    if (s != CL_OK) return s;
    float* Yd = S->Td;  // reuse the target buffer for the outputs
    cudaMemcpyAsync(S->Xd, X, sizeof(float) * n * S->n_in, cudaMemcpyHostToDevice, S->stream);
    for (int64_t r0 = 0; r0 < n; r0 += S->Bp) {
        const int nb = (int)std::min<int64_t>(S->Bp, n - r0);
        forward(S, nullptr, r0, nb, false);
        cl::destandardize_kernel<<<S->sms * 2, 256, 0, S->stream>>>(S->Z[S->L - 1], S->P[S->L], nb, S->n_out, S->mu_out,
                                                                    S->sd_out, Yd + r0 * S->n_out);
    }
    cudaMemcpyAsync(Y, Yd, sizeof(float) * n * S->n_out, cudaMemcpyDeviceToHost, S->stream);
    cudaError_t e = cudaStreamSynchronize(S->stream);
    return e == cudaSuccess ? check_tc(S, "surrogate_predict")
                            : sfail(CL_ERR_CUDA, std::string("surrogate_predict: ") + cudaGetErrorString(e));
}

}  // extern "C"
