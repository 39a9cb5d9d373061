// Internal declarations of the GB300 lattice library (not part of the ABI).
//
// State layout in HBM: every real field is split into a double-precision
// homogeneous mean (held in DevState) and a fluctuation array of N^3 values
// of type T (float or double), SoA, site index (z*N + y)*N + x.  Stencil
// passes read one copy of the arrays and write the other (ping-pong), so a
// pass never overwrites a value a neighbouring block still has to read.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is resolved through the runtime, no driver link)
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cl_lattice.h"

namespace cl {

constexpr int kMaxComp = 4;   // real components per sector (scalar fields, or Re/Im)
constexpr int kMaxSums = 48;  // reductions per pass
constexpr int kMaxArrays = 40;  // stored arrays per copy (SU(2) x U(1) + chi: 37)
constexpr int kMaxBlocks = 4096;

// Background, means and bookkeeping shared by all passes; lives in device
// memory and is updated by the last block of each pass (all FP64).
// DevState::error value of a pass whose tensor copies did not land within its wait limit
constexpr int kErrCopyTimeout = 1001;

struct DevState {
    double a;        // scale factor at the fields' time (where the next kick is evaluated)
    double b;        // a' (synchronized for VV; at the momenta's half step for LF)
    double bh;       // b_{1/2} carried between the two half kicks of a VV sub-step
    double t;        // program time of the fields
    double cd;       // drift coefficient of the next pass for scalar fields: w dt a_{1/2}^{-(3-alpha)}
    double cdA;      // drift coefficient of the next pass for link angles: e dx w dt a_{1/2}^{-(1-alpha)}
    double A1, A3, Am;  // a^{1+alpha}, a^{3+alpha}, a^{alpha-1} at the kick
    double EKm, EKAm;   // leapfrog: kinetic energies (field, gauge) at the previous half step
    double ahm;         // leapfrog: a at the previous half step
    double EGm, EVm, EGAm;  // leapfrog: gradient/potential/magnetic energies at the previous integer step
    double phibar[kMaxComp], pibar[kMaxComp];  // homogeneous means
    double sphi[kMaxComp], spi[kMaxComp];      // pending shifts: subtract from the stored arrays on read
    double E[8];        // energies of the last pass: scalar {EK0,EK1,EG0,EG1,EV1,EV2}; U(1) {EKp,EGp,EV,EKA,EGA}
    double sums[kMaxSums];  // normalized sums of the last pass
    double hc;          // Hubble-constraint violation of the last synchronized point
    double gauss[3];    // <G^2>, <lhs^2>, <rhs^2> of the last Gauss check
    double rk[4];       // RK4 / Gauss-Legendre: a and b at the step's start (RK4: and their stage sums)
    double gl_Da[2][5], gl_Db[2][5];  // Gauss-Legendre: scalar stage derivatives (two buffers)
    int gl_cur, gl_conv, gl_it;       // latest buffer, converged flag, sweeps of this step
    long long step;
    int error;          // nonzero: a reduction saw NaN/Inf, (CL_ERR_TIMEOUT) a Gauss-Legendre
                        // step did not converge, or (kErrCopyTimeout) a pass gave up waiting
                        // for its tensor copies; evolution stops
    int staggered;      // leapfrog momenta live half a step behind the fields
};

// What the last block does with the sums of a pass.
enum PassKind : int {
    PK_VV_FIRST = 0,   // first kick of a VV evolve call (no drift before it)
    PK_VV_MID = 1,     // merged kick between two VV sub-steps
    PK_VV_LAST = 2,    // closing half kick
    PK_LF = 3,         // leapfrog: kick, Friedmann fixed point, next drift
    PK_LF_PREPARE = 4, // backward half kick starting the leapfrog
    PK_MEASURE = 5,    // reductions only
    PK_INIT_B = 6,     // reductions only, then b from the Hubble constraint
    PK_LF_EKM = 7      // reductions only: E_K of the half-step-behind momenta
};

struct PassInfo {
    int kind;
    int pad;
    double dt;      // time step
    double wc, wn;  // weight of the sub-step just completed / of the next one
    double h1, h;   // kick of the energy evaluation / of the stored momenta
};

struct ModelConst {
    int kind, nf, pexp, N;
    double alpha, fmp2, lam, q, vev2, e, kappa, dx, idx2;
    // prescribed background (section 4.1): a(t) = bg_a0 (1 + bg_H0 t / bg_p)^bg_p when bg != 0
    int bg;
    double bg_p, bg_H0, bg_a0;
    int gpot;  // charged-scalar potential of the gauge models (cl_gauge_potential)
    // SU(2) x U(1) + chi: U(1) coupling of the doublet (0: none), singlet present,
    // and ext = either of the two (the 37-array layout)
    double e2;
    int chi, ext;
    int nc;  // U(1): non-compact gauge kinetics (section 5.2)
    // host-computed factors of the FP64 background update (one thread on the
    // device, where every division is a long dependent chain)
    double fmp2_3;      // (f*/m_p)^2 / 3
    double inv_vol;     // 1 / N^3
    double inv_e_sq;    // 1 / e^2 (gauge models)
    double inv_e2_sq;   // 1 / e_A^2 (SU(2) x U(1); 0 without the U(1) sector)
    double inv_dx4;     // 1 / dx^4
};

// Potential of the charged scalar of the gauge models as a function of
// mod2 = |phi|^2 (U(1)) or Phi^dag Phi (SU(2)), with *dv = dV/d(mod2), so that
// the force on phi is -dv phi: (lam/4)(mod2 - v2)^2 (sections 5, 6) or the
// monomial (lam/p)(2 mod2)^(p/2) with p = 2, 4, 6 (section 8).
template <class T>
__host__ __device__ inline T gauge_pot(int gpot, int p, T lam, T v2, T mod2, T* dv) {
    if (gpot == 0) {
        *dv = T(0.5) * lam * (mod2 - v2);
        return T(0.25) * lam * (mod2 - v2) * (mod2 - v2);
    }
    const T s = T(2) * mod2;
    T sp = T(1);  // s^(p/2 - 1)
    for (int k = 2; k < p; k += 2) sp *= s;
    *dv = lam * sp;
    return lam / T(p) * sp * s;
}

// d^2V/d(mod2)^2 of gauge_pot.
inline double gauge_pot_d2(int gpot, int p, double lam, double mod2) {
    if (gpot == 0) return 0.5 * lam;
    double sp = 1.0;  // (2 mod2)^(p/2 - 2)
    for (int k = 4; k < p; k += 2) sp *= 2.0 * mod2;
    return p > 2 ? lam * (p - 2) * sp : 0.0;
}

// Curvature of the potential along a canonical real component chi of the
// charged scalar (the squared canonical norm being 2 mod2):
// dV/dmod2 + chi^2 d^2V/dmod2^2.
inline double gauge_curvature(int gpot, int p, double lam, double v2, double mod2, double chi) {
    double dv;
    gauge_pot<double>(gpot, p, lam, v2, mod2, &dv);
    return dv + chi * chi * gauge_pot_d2(gpot, p, lam, mod2);
}

// x^e for x > 0.  When 2e is an integer with |2e| <= 32 (the program-unit
// exponents for alpha = 0, 1/2, 1, 3/2, ... and the a^4, a^6 of the energies)
// the power is formed from sqrt(x) and at most ten multiplications, a few ulp
// from the correctly rounded value; other exponents take pow.  The FP64 scalar
// updates of the passes run in one thread, where this is several times faster
// than pow.
__host__ __device__ inline double apow(double x, double e) {
    const double t = 2.0 * e;
    if (t == rint(t) && fabs(t) <= 32.0) {
        int n = (int)t;
        const bool inv = n < 0;
        if (inv) n = -n;
        double r = (n & 1) ? sqrt(x) : 1.0;
        double q = x;
        for (int m = n >> 1; m > 0; m >>= 1) {
            if (m & 1) r *= q;
            q *= q;
        }
        return inv ? 1.0 / r : r;
    }
    return pow(x, e);
}

// Scale factor and its program-time derivative of the prescribed background.
__host__ __device__ inline double bg_a(const ModelConst& mc, double t) {
    return mc.bg_a0 * apow(1.0 + mc.bg_H0 * t / mc.bg_p, mc.bg_p);
}
__host__ __device__ inline double bg_b(const ModelConst& mc, double t) {
    return mc.bg_a0 * mc.bg_H0 * apow(1.0 + mc.bg_H0 * t / mc.bg_p, mc.bg_p - 1.0);
}

// Per-lattice device resources.
struct Buffers {
    void* f[2][kMaxArrays];  // ping-pong copies of every stored array (type T)
    int narr;
    DevState* st;
    double* partials;  // per-block partial sums
    unsigned int* counter;
};

// Tile geometry of the stencil passes.
struct Geometry {
    int N, V, BX, BY, ZC, S;  // S: stages of the shared-memory plane ring
    int ntx, nty, ntz, ntiles, grid, threads;
    size_t smem;
};

// Host-side handle.
struct Lattice {
    ModelConst mc;
    cl_grid grid;
    cl_init init;
    int integ;
    int prec;  // CL_FP64 / CL_FP32
    size_t tsize;
    cudaStream_t stream;
    Buffers buf;
    int cur;   // which ping-pong copy holds the current state
    Geometry geo;
    std::vector<double> weights;
    long long steps_done;
    std::string err;
    // graphs cached by (steps, parity)
    struct G { long long steps; int parity; int part; int end_parity; cudaGraphExec_t exec; };
    std::vector<G> graphs;
    cufftHandle plan_c2r, plan_r2c;
    bool plans;
    double* work;      // FP64 scratch of N^3 (conversion, spectra)
    void* cwork;       // complex FP64 scratch N*N*(N/2+1) (x2)
    double* bins;      // spectrum accumulators
    int sm_count;
    cudaStream_t cstream;  // private stream used only to record graphs
    bool staggered;        // host mirror of DevState::staggered
    bool shared_fft;       // plans and FFT scratch belong to an ensemble
    void* rk_T1[4];        // RK4: second stage copy (the first is the spare ping-pong copy)
    void* rk_A[4];         // RK4: accumulator
    void* gl_D[2][5][4];   // Gauss-Legendre: stage derivatives, two buffers
};

// cuFFT plans and FP64 scratch that the members of an ensemble of one lattice size share.
struct SharedFFT {
    cufftHandle c2r, r2c;
    double* work;
    void* cwork;
};

// lattice_init with optional shared FFT resources (lattice_api.cu).
cl_status lattice_create(const cl_model* model, const cl_grid* grid, const cl_init* init, cudaStream_t stream,
                         const SharedFFT* shared, cl_lattice** out);
void set_global_error(const char* msg);
// Tensor map of one N^3 array of element size tsize (x fastest) for boxes of
// bx x by x 1 elements (one z plane); no interleave, swizzle or out-of-range
// fill beyond the default zeros.  false when the encoder is unavailable or
// rejects the box.
bool encode_plane_box(CUtensorMap* map, const void* base, int N, size_t tsize, int bx, int by);

// ---- device helpers -------------------------------------------------------

template <typename T> struct VecT;
template <> struct VecT<float> { using type = float4; static constexpr int V = 4; };
template <> struct VecT<double> { using type = double2; static constexpr int V = 2; };

__device__ __forceinline__ void vload(const float* p, float (&r)[4]) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
}
__device__ __forceinline__ void vload(const double* p, double (&r)[2]) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    r[0] = v.x; r[1] = v.y;
}
__device__ __forceinline__ void vload_s(const float* p, float (&r)[4]) {
    float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
}
__device__ __forceinline__ void vload_s(const double* p, double (&r)[2]) {
    double2 v = *reinterpret_cast<const double2*>(p);
    r[0] = v.x; r[1] = v.y;
}
__device__ __forceinline__ void vstore(float* p, const float (&r)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void vstore(double* p, const double (&r)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
}
__device__ __forceinline__ void vstore_cs(float* p, const float (&r)[4]) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(r[0], r[1], r[2], r[3]));
}
__device__ __forceinline__ void vstore_cs(double* p, const double (&r)[2]) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(r[0], r[1]));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the nl existing lanes of a possibly partial warp (nl = 1..32);
// the result is valid in lane 0.  Shuffles name only existing lanes.
// One warp's compensated sum of partials[b * ns + s] over b < nb: lane l takes
// b = l, l + nl, ... in that order into a Kahan accumulator (Kahan 1965), with
// the loads issued eight at a time so that their L2 latencies overlap; a
// shuffle tree then adds the lanes' compensated sums.  The order is fixed, so
// every run gives the same bits.  (The cost is set by GB300's FP64 throughput:
// four FP64 operations per partial.)
__device__ __forceinline__ double warp_partials_sum(const double* partials, int nb, int ns, int s, int lane, int nl) {
    double ks = 0.0, kc = 0.0;
    for (int b0 = lane; b0 < nb; b0 += 8 * nl) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int b = b0 + k * nl;
            v[k] = b < nb ? __ldcg(&partials[(size_t)b * ns + s]) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (b0 + k * nl < nb) {
                const double yk = v[k] - kc, tk = ks + yk;
                kc = (tk - ks) - yk;
                ks = tk;
            }
        }
    }
    double acc = ks - kc;
    const unsigned mask = nl >= 32 ? 0xffffffffu : ((1u << nl) - 1u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_down_sync(mask, acc, o);
        if (lane + o < nl) acc += t;
    }
    return acc;
}

// Adds the per-thread sums ts[0..NS-1] of a warp into the warp's FP64
// accumulators acc[0..NS-1] and clears ts.  Full warps use a butterfly whose
// every exchange halves the values a lane carries (16 -> 8 -> 4 -> 2 -> 1;
// 16 shuffles in all instead of 5 per sum); lane 2s then holds the warp total
// of sum s = lane/2.  The order of additions is fixed, so results repeat bit
// for bit.  Partial warps take one shuffle tree per sum.
template <typename T, int NS>
__device__ __forceinline__ void fold_warp_sums(T (&ts)[NS], double* acc, int lane, int nlanes) {
    static_assert(NS <= 16, "at most 16 sums per fold");
    if (nlanes == 32) {
        // in place on ts; entries at and beyond NS count as zero
#pragma unroll
        for (int w = 8, o = 16; w >= 1; w >>= 1, o >>= 1) {
            const bool hi = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < w; ++j) {
                if (j >= NS) continue;
                const T lo_v = ts[j], hi_v = (j + w < NS) ? ts[j + w] : T(0);
                const T send = hi ? lo_v : hi_v;
                const T keep = hi ? hi_v : lo_v;
                ts[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        ts[0] += __shfl_xor_sync(0xffffffffu, ts[0], 1);
        const int s = lane >> 1;
        if ((lane & 1) == 0 && s < NS) acc[s] += double(ts[0]);
    } else {
        const unsigned mask = (1u << nlanes) - 1u;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            T v = ts[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T t = __shfl_down_sync(mask, v, o);
                if (lane + o < nlanes) v += t;
            }
            if (lane == 0) acc[i] += double(v);
        }
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) ts[i] = T(0);
}

template <typename T> __device__ __forceinline__ T partial_warp_sum(T v, int lane, int nl) {
    const unsigned mask = nl >= 32 ? 0xffffffffu : ((1u << nl) - 1u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T t = __shfl_down_sync(mask, v, o);
        if (lane + o < nl) v += t;
    }
    return v;
}

// ---- bulk-async copies and mbarriers (inline PTX, sm_90+ / sm_103a) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait that may suspend the thread (it issues nothing meanwhile) until the
// phase completes or about `ns` nanoseconds pass
__device__ __forceinline__ bool mbar_try_wait_for(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// The same wait with a time limit (about 2 s of SM clock); false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded_sleep(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait_for(bar, parity, 1000000u)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait_for(bar, parity, 1000000u))
        if (clock64() - t0 > 4000000000LL) return false;
    return true;
}
// Wait for a phase with a time limit (about 2 s of SM clock); false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > 4000000000LL) return false;
    return true;
}
// Tiled tensor copy of one box of a 3-D map (x, y, z) into shared memory,
// completion counted in bytes on the mbarrier.  The map lives in kernel
// parameter space (a __grid_constant__ argument); the destination is this
// CTA's shared memory, 128-byte aligned; x times the element size is a
// multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
// Hint: bring the line holding p into L2 (no register result, no fault semantics
// needed: callers only pass addresses inside their arrays).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// Per-thread asynchronous global -> shared copies (16 bytes, or 4/8 bytes for halo cells).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* dst, const double* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC11 2011): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint32_t lo0 = M0 * c[0], hi0 = __umulhi(M0, c[0]);
        const uint32_t lo1 = M1 * c[2], hi1 = __umulhi(M1, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// ---- host entry points between translation units --------------------------

// scalar_pass.cu
cudaError_t scalar_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s);
cudaError_t scalar_launch_drift(Lattice* L, int cur, cudaStream_t s);  // leapfrog closing drift (in place)
void scalar_geometry(Lattice* L);

// rk4.cu: m explicit RK4 steps of the state in copy `cur` (FP64 scalar model)
cudaError_t rk4_enqueue(Lattice* L, long long m, int cur, cudaStream_t s);
// gl.cu: m Gauss-Legendre steps of the state in copy `cur` (FP64 scalar model)
cudaError_t gl_enqueue(Lattice* L, long long m, int cur, cudaStream_t s);

// u1_pass.cu
cudaError_t u1_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s);
cudaError_t u1_launch_drift(Lattice* L, int cur, cudaStream_t s);
cudaError_t u1_launch_gauss(Lattice* L, int cur, cudaStream_t s);
void u1_geometry(Lattice* L);

// su2_pass.cu
cudaError_t su2_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s);
cudaError_t su2_launch_drift(Lattice* L, int cur, cudaStream_t s);
cudaError_t su2_launch_gauss(Lattice* L, int cur, cudaStream_t s);
cudaError_t su2_fill(Lattice* L, const double* phi, const double* pi);
void su2_geometry(Lattice* L);

// ic.cu
cl_status ic_generate(Lattice* L);
cudaError_t launch_finish_drift(Lattice* L, cudaStream_t s);

// fields.cu
cudaError_t launch_get_field(Lattice* L, int which, double* dst, cudaStream_t s);
cudaError_t launch_set_field(Lattice* L, int which, const double* src, cudaStream_t s);
cudaError_t launch_get_stored(Lattice* L, int slot, void* dst, double* mean_dev, cudaStream_t s);
cudaError_t launch_set_stored_mean(Lattice* L, int slot, double mean, cudaStream_t s);
int has_mean(const ModelConst& mc, int slot);
cudaError_t launch_spectrum(Lattice* L, int slot, int accumulate, cudaStream_t s);
// Gauge-field spectra: sector 0 U(1), 1 SU(2); what 0 electric momenta, 1 magnetic
// field; accumulates every component into L->bins and returns their number.
cudaError_t launch_gauge_spectrum(Lattice* L, int sector, int what, int* ncomp, cudaStream_t s);
int spectrum_bins(int N);

// ensemble.cu: the CL_OBS_SIZE observables of a two-field lattice from its
// measured state and chi shell sums (3 x spectrum_bins(N) doubles)
void observables(const DevState& s, const double* bins, int N, double dx, double kIR, double kmax, float* o);

int array_count(const ModelConst& mc);
int array_slot(const ModelConst& mc, int which);  // ABI index -> storage slot, -1 if invalid

}  // namespace cl
