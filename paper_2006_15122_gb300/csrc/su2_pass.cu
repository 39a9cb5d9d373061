// SU(2)-Higgs sector (paper section 6): a complex doublet Phi with momentum
// pi = a^{3-alpha} Phi', links U_i = exp(-i g dx B_i^a sigma^a/2) stored as
// unit quaternions U = q0 + i q.sigma (SU(2) toolkit, section 3.2.3), and
// electric momenta piB_i^a = a^{1-alpha} G_0i^a.
//
// Kernels (section 6.2), from the gauge-invariant lattice Hamiltonian built on
// the energies of section 6.3.1 (kappa = (w*/f*)^2, g = g_B Q_B):
//   K_Phi    = -a^{3+alpha} (lam/2)(|Phi|^2 - v2) Phi
//              + a^{1+alpha} sum_i (U_i Phi(n+i) - 2 Phi + U_i^dag(n-i) Phi(n-i)) / dx^2,
//   K_B,i^a  = a^{1+alpha} (g/(kappa dx)) Im[Phi^dag sigma^a U_i Phi(n+i)]
//              + a^{alpha-1} (2/(g dx^3)) sum_{j!=i} (P_a[U_ij(n)] - P_a[U_j^dag(n-j) U_ij(n-j) U_j(n-j)]),
//   U_ij(n)  = U_i(n) U_j(n+i) U_i^dag(n+j) U_j^dag(n),  P_a[q] = q_a,
// drifts phi += c pi, U_i <- exp(-i c' piB_i^a sigma^a/2) U_i (exact exponential,
// unit quaternions renormalised), and the discrete Gauss law
//   (1/dx) sum_i [piB_i(n) - U_i^dag(n-i) piB_i(n-i) U_i(n-i)]^a = (g/kappa) Im[Phi^dag sigma^a pi].
//
// One pass = a drift kernel (src copy -> dst copy, pointwise) followed by a
// kick kernel in place on dst (stencil through L1/L2), which also reduces the
// volume sums and runs the FP64 background update in its last block, shared
// with the U(1) sector.  Array slots: 0-3 Phi (Re/Im of the two components),
// 4-7 pi, 8-19 links (4 i + c), 20-28 piB (3 i + a).
//
// SU(2) x U(1) + chi (section 8.3; the EXT kernels): the doublet also carries
// a U(1) charge eA (link angles theta_i, V_i = exp(-i theta_i), electric
// momenta piA_i; slots 29-31, 32-34) and couples to a real singlet chi (slots
// 35, 36) through V_int = q |Phi|^2 chi^2.  The transporter of Phi becomes
// W_i = V_i U_i, and
//   K_Phi  = -a^{3+alpha}(V' + q chi^2) Phi + a^{1+alpha} sum_i (W_i Phi(n+i) - 2 Phi + W_i^dag(n-i) Phi(n-i))/dx^2,
//   K_B    as above with W_i Phi(n+i) in the current,
//   K_A,i  = a^{1+alpha}(2 eA/(kappa dx)) Im[Phi^dag W_i Phi(n+i)]
//            + a^{alpha-1}/(eA dx^3) sum_{j!=i} [sin theta_ij(n-j) - sin theta_ij(n)],
//   K_chi  = -a^{3+alpha} 2 q |Phi|^2 chi + a^{1+alpha} L[chi],
// theta_ij(n) = theta_i(n) + theta_j(n+i) - theta_i(n+j) - theta_j(n); the U(1)
// Gauss law is (1/dx) sum_i [piA_i(n) - piA_i(n-i)] = (2 eA/kappa) Im[Phi^dag pi].
// Four more volume sums (sync piA^2, sum_{i<j} (1 - cos theta_ij), sync pchi^2,
// grad chi^2) enter the shared background update.
#include <math.h>

#include "cl_internal.cuh"
#include "gauge_finish.cuh"

namespace cl {

constexpr int kSu2Arrays = 37;  // 29 without the U(1) sector and the singlet
constexpr int kSu2ExtNS = 15;   // volume sums of the EXT kernels

struct Su2Args {
    void* a[kSu2Arrays];  // kick: the copy updated in place
    DevState* st;
    double* partials;
    unsigned int* counter;
    ModelConst mc;
    PassInfo pi;
    int write;
};

template <typename T> __device__ __forceinline__ void qmul(const T* p, const T* q, T* r) {
    const T r0 = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
    const T r1 = p[0] * q[1] + q[0] * p[1] - (p[2] * q[3] - p[3] * q[2]);
    const T r2 = p[0] * q[2] + q[0] * p[2] - (p[3] * q[1] - p[1] * q[3]);
    const T r3 = p[0] * q[3] + q[0] * p[3] - (p[1] * q[2] - p[2] * q[1]);
    r[0] = r0; r[1] = r1; r[2] = r2; r[3] = r3;
}
template <typename T> __device__ __forceinline__ void qconj(const T* q, T* r) {
    r[0] = q[0]; r[1] = -q[1]; r[2] = -q[2]; r[3] = -q[3];
}
// U Phi, U = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
template <typename T> __device__ __forceinline__ void umul(const T* q, const T* f, T* o) {
    o[0] = q[0] * f[0] - q[3] * f[1] + q[2] * f[2] - q[1] * f[3];
    o[1] = q[0] * f[1] + q[3] * f[0] + q[2] * f[3] + q[1] * f[2];
    o[2] = -q[2] * f[0] - q[1] * f[1] + q[0] * f[2] + q[3] * f[3];
    o[3] = -q[2] * f[1] + q[1] * f[0] + q[0] * f[3] - q[3] * f[2];
}
// Im[x^dag sigma^a y], a = 1..3
template <typename T> __device__ __forceinline__ void im_sigma(const T* x, const T* y, T* o) {
    o[0] = x[0] * y[3] - x[1] * y[2] + x[2] * y[1] - x[3] * y[0];
    o[1] = -x[0] * y[2] - x[1] * y[3] + x[2] * y[0] + x[3] * y[1];
    o[2] = x[0] * y[1] - x[1] * y[0] - x[2] * y[3] + x[3] * y[2];
}

__device__ __forceinline__ void half_sincos(float t, float* s, float* c) { sincosf(0.5f * t, s, c); }
__device__ __forceinline__ void half_sincos(double t, double* s, double* c) { sincos(0.5 * t, s, c); }

// U(1) phases: FP32 takes the hardware approximation on wrapped angles (sums of
// at most four angles in [-pi, pi]), as the compact U(1) sector does
__device__ __forceinline__ void phase_sc(float t, float* s, float* c) { __sincosf(t, s, c); }
__device__ __forceinline__ void phase_sc(double t, double* s, double* c) { sincos(t, s, c); }
template <typename T> __device__ __forceinline__ T wrap_phase(T t) {
    const T twopi = T(6.283185307179586476925287);
    return t - twopi * rint(t / twopi);
}
// (a + i b) -> e^{-i t}(a + i b) on both components of a doublet, given (sin t, cos t)
template <typename T> __device__ __forceinline__ void phase_minus(T* v, T s, T c) {
    const T v0 = c * v[0] + s * v[1], v1 = c * v[1] - s * v[0];
    const T v2 = c * v[2] + s * v[3], v3 = c * v[3] - s * v[2];
    v[0] = v0; v[1] = v1; v[2] = v2; v[3] = v3;
}
template <typename T> __device__ __forceinline__ void phase_plus(T* v, T s, T c) { phase_minus(v, -s, c); }
// Im[x^dag y] for doublets
template <typename T> __device__ __forceinline__ T im_dot(const T* x, const T* y) {
    return x[0] * y[1] - x[1] * y[0] + x[2] * y[3] - x[3] * y[2];
}

template <typename T> __device__ __forceinline__ void ldq(T* const* a, int i, size_t n, T* q) {
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = __ldg(a[8 + 4 * i + c] + n);
}
template <typename T> __device__ __forceinline__ void ldf(T* const* a, size_t n, T* f) {
#pragma unroll
    for (int c = 0; c < 4; ++c) f[c] = __ldg(a[c] + n);
}

template <typename T> __device__ __forceinline__ size_t nb(size_t n, int x, int y, int z, int N, int d, int s) {
    const size_t NN = (size_t)N * N;
    if (d == 0) {
        const int xx = x + s < 0 ? x + s + N : (x + s >= N ? x + s - N : x + s);
        return n - x + xx;
    }
    if (d == 1) {
        const int yy = y + s < 0 ? y + s + N : (y + s >= N ? y + s - N : y + s);
        return n + (size_t)(yy - y) * N;
    }
    const int zz = z + s < 0 ? z + s + N : (z + s >= N ? z + s - N : z + s);
    return n + (size_t)(zz - z) * NN;
}

// plaquette U_ij at site m (coordinates x, y, z)
template <typename T>
__device__ __forceinline__ void plaq(T* const* a, int i, int j, size_t m, int x, int y, int z, int N, T* P) {
    T Ui[4], Ujp[4], Uip[4], Uj[4], t1[4], t2[4], c[4];
    ldq(a, i, m, Ui);
    ldq(a, j, nb<T>(m, x, y, z, N, i, 1), Ujp);
    ldq(a, i, nb<T>(m, x, y, z, N, j, 1), Uip);
    ldq(a, j, m, Uj);
    qmul(Ui, Ujp, t1);
    qconj(Uip, c);
    qmul(t1, c, t2);
    qconj(Uj, c);
    qmul(t2, c, P);
}

// backward staple of link i at n in the plane (i, j), transported to n:
// U_j^dag(n-j) U_ij(n-j) U_j(n-j) = U_j^dag(n-j) U_i(n-j) U_j(n-j+i) U_i^dag(n),
// the two factors U_j^dag(n-j) U_j(n-j) = 1 of the plaquette form cancelled
// (unit links); uic = U_i^dag(n)
template <typename T>
__device__ __forceinline__ void back_staple(T* const* a, int i, int j, size_t n, int x, int y, int z, int N,
                                            const T* uic, T* Q) {
    const size_t mj = nb<T>(n, x, y, z, N, j, -1);
    const int xj = j == 0 ? (x == 0 ? N - 1 : x - 1) : x;
    const int yj = j == 1 ? (y == 0 ? N - 1 : y - 1) : y;
    const int zj = j == 2 ? (z == 0 ? N - 1 : z - 1) : z;
    T Uj[4], Ui[4], Ujp[4], c[4], t1[4], t2[4];
    ldq(a, j, mj, Uj);
    ldq(a, i, mj, Ui);
    ldq(a, j, nb<T>(mj, xj, yj, zj, N, i, 1), Ujp);
    qconj(Uj, c);
    qmul(c, Ui, t1);
    qmul(t1, Ujp, t2);
    qmul(t2, uic, Q);
}

template <typename T, bool EXT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) su2_kick_kernel(const Su2Args A) {
    constexpr int NS = EXT ? kSu2ExtNS : U1NS;
    DevState* st = A.st;
    if (st->error) return;
    const int N = A.mc.N;
    T* const* arr = reinterpret_cast<T* const*>(A.a);
    const T A1 = T(st->A1), A3 = T(st->A3), Am = T(st->Am);
    const T h1 = T(A.pi.h1), h = T(A.pi.h), idx2 = T(A.mc.idx2);
    const T lam = T(A.mc.lam), v2 = T(A.mc.vev2);
    const T cJ = T(A.mc.e / (A.mc.kappa * A.mc.dx)), cM = T(2.0 / (A.mc.e * A.mc.dx * A.mc.dx * A.mc.dx));
    const bool hasA = EXT && A.mc.e2 > 0, hasC = EXT && A.mc.chi;
    const T cJA = hasA ? T(2.0 * A.mc.e2 / (A.mc.kappa * A.mc.dx)) : T(0);
    const T cMA = hasA ? T(1.0 / (A.mc.e2 * A.mc.dx * A.mc.dx * A.mc.dx)) : T(0);
    const T qc = T(A.mc.q);
    const size_t n3 = (size_t)N * N * N;
    // per-thread sums in T, folded into FP64 every 64 sites
    double acc[NS];
    T ts[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) { acc[s] = 0.0; ts[s] = T(0); }
    int cnt = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < n3; n += stride) {
        // the grid's next chunk of sites into L2 while this one computes: its loads
        // (own sites and most neighbours) then wait on L2, not on DRAM
        if (n + stride < n3) {
#pragma unroll
            for (int a = 0; a < (EXT ? 37 : 29); ++a)
                if (a < 29 || (a < 35 ? hasA : hasC)) prefetch_l2(arr[a] + n + stride);
        }
        const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / ((size_t)N * N));
        T f[4], lap[4], grad = T(0), eB = T(0);
        ldf(arr, n, f);
#pragma unroll
        for (int c = 0; c < 4; ++c) lap[c] = T(-6) * f[c];
        T KB[3][3];
        // U(1) sector: forward plaquette angles theta_01, theta_02, theta_12 at n (sines, cosines)
        T KA[3] = {T(0), T(0), T(0)}, eBA = T(0), chi0 = T(0), lchi = T(0), gchi = T(0);
        T psn[3] = {T(0), T(0), T(0)};
        if (hasA) {
            T th0[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) th0[d] = arr[29 + d][n];
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
                const int ii = pr == 2 ? 1 : 0, jj = pr == 0 ? 1 : 2;
                const T p = th0[ii] + arr[29 + jj][nb<T>(n, x, y, z, N, ii, 1)] - arr[29 + ii][nb<T>(n, x, y, z, N, jj, 1)] -
                            th0[jj];
                T cs;
                phase_sc(p, &psn[pr], &cs);
                eBA += T(1) - cs;
            }
        }
        if (hasC) chi0 = arr[35][n];
        // forward plaquettes U_01, U_02, U_12 at n: vector parts and magnetic energy
        // (U_ji = U_ij^dag, so the plane (j, i) takes the vector part with the sign flipped)
        T Pv[3][3];
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
            const int ii = pr == 2 ? 1 : 0, jj = pr == 0 ? 1 : 2;
            T P[4];
            plaq(arr, ii, jj, n, x, y, z, N, P);
            eB += T(4) * (T(1) - P[0]);
#pragma unroll
            for (int k = 0; k < 3; ++k) Pv[pr][k] = P[k + 1];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const size_t np = nb<T>(n, x, y, z, N, i, 1), nm = nb<T>(n, x, y, z, N, i, -1);
            T q[4], qm[4], c[4], fp[4], fm[4], t[4], t2[4];
            ldq(arr, i, n, q);
            ldq(arr, i, nm, qm);
            qconj(qm, c);
            ldf(arr, np, fp);
            ldf(arr, nm, fm);
            umul(q, fp, t);
            umul(c, fm, t2);
            if (hasA) {  // W_i Phi(n+i) = e^{-i theta_i(n)} U_i Phi(n+i); W_i^dag(n-i) = U^dag e^{+i theta_i(n-i)}
                T sn, cs;
                phase_sc(arr[29 + i][n], &sn, &cs);
                phase_minus(t, sn, cs);
                phase_sc(arr[29 + i][nm], &sn, &cs);
                phase_plus(t2, sn, cs);
            }
            if (hasC) {
                const T cp = arr[35][np];
                lchi += cp + arr[35][nm];
                gchi += (cp - chi0) * (cp - chi0);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                lap[k] += t[k] + t2[k];
                grad += (t[k] - f[k]) * (t[k] - f[k]);
            }
            T js[3];
            im_sigma(f, t, js);
            T mag[3] = {T(0), T(0), T(0)};
            T uic[4];
            qconj(q, uic);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (j == i) continue;
                const int pr = i + j - 1;  // (0,1) -> 0, (0,2) -> 1, (1,2) -> 2
                const T sg = i < j ? T(1) : T(-1);
                T Q[4];
                back_staple(arr, i, j, n, x, y, z, N, uic, Q);
#pragma unroll
                for (int k = 0; k < 3; ++k) mag[k] += sg * Pv[pr][k] - Q[k + 1];
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) KB[i][k] = A1 * cJ * js[k] + Am * cM * mag[k];
            if (hasA) {
                // sum_{j != i} [sin theta_ij(n-j) - sin theta_ij(n)], theta_ji = -theta_ij
                T magA = T(0);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (j == i) continue;
                    const int ii = i < j ? i : j, jj = i < j ? j : i;
                    const T sgn = i < j ? T(1) : T(-1);
                    const size_t mj = nb<T>(n, x, y, z, N, j, -1);
                    const int xj = j == 0 ? (x == 0 ? N - 1 : x - 1) : x;
                    const int yj = j == 1 ? (y == 0 ? N - 1 : y - 1) : y;
                    const int zj = j == 2 ? (z == 0 ? N - 1 : z - 1) : z;
                    // theta_ij(n-j) = theta_i(n-j) + theta_j(n-j+i) - theta_i(n) - theta_j(n-j)
                    const T pm = arr[29 + i][mj] + arr[29 + j][nb<T>(mj, xj, yj, zj, N, i, 1)] - arr[29 + i][n] -
                                 arr[29 + j][mj];
                    T smm, cmm;
                    phase_sc(pm, &smm, &cmm);
                    magA += smm - sgn * psn[ii + jj - 1];
                }
                KA[i] = A1 * cJA * im_dot(f, t) + Am * cMA * magA;
            }
        }
        const T mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];
        T dv;
        T vpot = gauge_pot<T>(A.mc.gpot, A.mc.pexp, lam, v2, mod2, &dv);
        if (hasC) {
            dv += qc * chi0 * chi0;
            vpot += qc * mod2 * chi0 * chi0;
        }
        T sp = T(0), pr0 = T(0), pr1 = T(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const T K = -A3 * dv * f[c] + A1 * lap[c] * idx2;
            const T p = arr[4 + c][n];
            const T ps = p + h1 * K;
            sp += ps * ps;
            if (c == 0) pr0 = ps;
            if (c == 1) pr1 = ps;
            if (A.write) arr[4 + c][n] = p + h * K;
        }
        T sA = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T e = arr[20 + 3 * i + k][n];
                const T es = e + h1 * KB[i][k];
                sA += es * es;
                if (A.write) arr[20 + 3 * i + k][n] = e + h * KB[i][k];
            }
        ts[0] += f[0]; ts[1] += f[1];
        ts[2] += f[0] * f[0]; ts[3] += f[1] * f[1];
        ts[4] += pr0; ts[5] += pr1;
        ts[6] += sp;
        ts[7] += grad * idx2;
        ts[8] += vpot;
        ts[9] += sA;
        ts[10] += eB;
        if (hasA) {
            T sAA = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T e = arr[32 + i][n];
                const T es = e + h1 * KA[i];
                sAA += es * es;
                if (A.write) arr[32 + i][n] = e + h * KA[i];
            }
            ts[11 % NS] += sAA;
            ts[12 % NS] += eBA;
        }
        if (hasC) {
            const T Kc = -A3 * T(2) * qc * mod2 * chi0 + A1 * (lchi - T(6) * chi0) * idx2;
            const T p = arr[36][n];
            const T ps = p + h1 * Kc;
            if (A.write) arr[36][n] = p + h * Kc;
            ts[13 % NS] += ps * ps;
            ts[14 % NS] += gchi * idx2;
        }
        if (++cnt == 64) {
#pragma unroll
            for (int s = 0; s < NS; ++s) { acc[s] += double(ts[s]); ts[s] = T(0); }
            cnt = 0;
        }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] += double(ts[s]);
    // block reduction, partials, last block
    __shared__ double red[8][NS];
    const int lin = threadIdx.x, lane = lin & 31, warp = lin >> 5, nwarps = (blockDim.x + 31) >> 5;
    const int nlanes = min(32, (int)blockDim.x - 32 * warp);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const double v = partial_warp_sum(acc[s], lane, nlanes);
        if (lane == 0) red[warp][s] = v;
    }
    __syncthreads();
    if (lin < NS) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += red[w][lin];
        A.partials[(size_t)blockIdx.x * NS + lin] = t;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int last;
    if (lin == 0) last = (atomicAdd(A.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[NS];
    const double invV = 1.0 / (double)n3;
    for (int s = warp; s < NS; s += nwarps) {
        double ks = 0.0, kc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += nlanes) {
            const double yk = __ldcg(&A.partials[(size_t)b * NS + s]) - kc, tk = ks + yk;
            kc = (tk - ks) - yk;
            ks = tk;
        }
        const double r = partial_warp_sum(ks - kc, lane, nlanes);
        if (lane == 0) tot[s] = r * invV;
    }
    __syncthreads();
    if (lin == 0) {
        *A.counter = 0u;
        u1_finish(st, tot, A.mc, A.pi, NS);
    }
}

// Drift with the coefficients prepared by the last pass: phi += cd pi,
// U_i <- exp(-i cdA piB_i.sigma/2) U_i (renormalised); momenta copied.
// EXT: also theta_i += (eA/g) cdA piA_i (wrapped to [-pi, pi]) and chi += cd pchi.
// src and dst may coincide (pointwise).
template <typename T, bool EXT>
__global__ void su2_drift_kernel(const Su2Args S, const Su2Args D) {
    const DevState* st = S.st;
    if (st->error) return;
    const T cd = T(st->cd), cU = T(st->cdA);
    const size_t n3 = (size_t)S.mc.N * S.mc.N * S.mc.N;
    T* const* src = reinterpret_cast<T* const*>(S.a);
    T* const* dst = reinterpret_cast<T* const*>(D.a);
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < n3; n += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const T p = src[4 + c][n];
            dst[c][n] = src[c][n] + cd * p;
            dst[4 + c][n] = p;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T e[3], q[4], ex[4], r[4];
#pragma unroll
            for (int k = 0; k < 3; ++k) e[k] = src[20 + 3 * i + k][n];
#pragma unroll
            for (int c = 0; c < 4; ++c) q[c] = src[8 + 4 * i + c][n];
            const T ex0 = cU * e[0], ex1 = cU * e[1], ex2 = cU * e[2];
            const T th = sqrt(ex0 * ex0 + ex1 * ex1 + ex2 * ex2);
            T s, c;
            half_sincos(th, &s, &c);
            const T sf = th > T(0) ? s / th : T(0.5);
            ex[0] = c; ex[1] = -sf * ex0; ex[2] = -sf * ex1; ex[3] = -sf * ex2;
            qmul(ex, q, r);
            const T nr = T(1) / sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) dst[8 + 4 * i + c2][n] = r[c2] * nr;
#pragma unroll
            for (int k = 0; k < 3; ++k) dst[20 + 3 * i + k][n] = e[k];
        }
        if (EXT) {
            const T cA = S.mc.e2 > 0 ? T(st->cdA * (S.mc.e2 / S.mc.e)) : T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T e = src[32 + i][n];
                dst[29 + i][n] = S.mc.e2 > 0 ? wrap_phase(src[29 + i][n] + cA * e) : src[29 + i][n];
                dst[32 + i][n] = e;
            }
            const T pc = src[36][n];
            dst[35][n] = src[35][n] + cd * pc;
            dst[36][n] = pc;
        }
    }
}

// Gauss residual G^a = (1/dx) sum_i [piB_i(n) - (U_i^dag(n-i) piB_i(n-i) U_i(n-i))]^a
//                      - (g/kappa) Im[Phi^dag sigma^a pi], FP64 sums into st->gauss;
// EXT with the U(1) sector adds G^0 = (1/dx) sum_i [piA_i(n) - piA_i(n-i)] - (2 eA/kappa) Im[Phi^dag pi].
template <typename T, bool EXT>
__global__ void su2_gauss_kernel(const Su2Args A) {
    const int N = A.mc.N;
    const size_t n3 = (size_t)N * N * N;
    T* const* arr = reinterpret_cast<T* const*>(A.a);
    const double idx = 1.0 / A.mc.dx, c = A.mc.e / A.mc.kappa;
    double g2 = 0, l2 = 0, r2 = 0;
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < n3; n += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / ((size_t)N * N));
        double div[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) {
            const size_t nm = nb<T>(n, x, y, z, N, i, -1);
            double q[4], qc[4], e[4], t[4], tr[4];
            for (int k = 0; k < 4; ++k) q[k] = (double)arr[8 + 4 * i + k][nm];
            qconj(q, qc);
            e[0] = 0.0;
            for (int k = 0; k < 3; ++k) e[k + 1] = (double)arr[20 + 3 * i + k][nm];
            qmul(qc, e, t);
            qmul(t, q, tr);
            for (int k = 0; k < 3; ++k) div[k] += ((double)arr[20 + 3 * i + k][n] - tr[k + 1]) * idx;
        }
        double f[4], p[4], rho[3];
        for (int k = 0; k < 4; ++k) {
            f[k] = (double)arr[k][n];
            p[k] = (double)arr[4 + k][n];
        }
        im_sigma(f, p, rho);
        for (int k = 0; k < 3; ++k) {
            const double r = c * rho[k];
            g2 += (div[k] - r) * (div[k] - r);
            l2 += div[k] * div[k];
            r2 += r * r;
        }
        if (EXT && A.mc.e2 > 0) {
            double d0 = 0.0;
            for (int i = 0; i < 3; ++i)
                d0 += ((double)arr[32 + i][n] - (double)arr[32 + i][nb<T>(n, x, y, z, N, i, -1)]) * idx;
            const double r = 2.0 * A.mc.e2 / A.mc.kappa * im_dot(f, p);
            g2 += (d0 - r) * (d0 - r);
            l2 += d0 * d0;
            r2 += r * r;
        }
    }
    g2 = warp_sum(g2);
    l2 = warp_sum(l2);
    r2 = warp_sum(r2);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&A.st->gauss[0], g2 / (double)n3);
        atomicAdd(&A.st->gauss[1], l2 / (double)n3);
        atomicAdd(&A.st->gauss[2], r2 / (double)n3);
    }
}

// Homogeneous initial state: Phi = phi0, pi = a^{3-alpha} dphi0, unit links, zero piB
// (and zero angles, piA, chi, pchi).
template <typename T>
__global__ void su2_fill_kernel(const Su2Args A, int narr, double f0, double f1, double f2, double f3, double p0,
                                double p1, double p2, double p3) {
    const size_t n3 = (size_t)A.mc.N * A.mc.N * A.mc.N;
    T* const* arr = reinterpret_cast<T* const*>(A.a);
    const double v[8] = {f0, f1, f2, f3, p0, p1, p2, p3};
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < n3; n += (size_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 8; ++k) arr[k][n] = T(v[k]);
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 4; ++c) arr[8 + 4 * i + c][n] = T(c == 0 ? 1.0 : 0.0);
        for (int k = 20; k < narr; ++k) arr[k][n] = T(0);
    }
}

__global__ void zero_su2_gauss_kernel(DevState* st) { st->gauss[0] = st->gauss[1] = st->gauss[2] = 0.0; }

static Su2Args su2_args(Lattice* L, int copy) {
    Su2Args A;
    for (int k = 0; k < kSu2Arrays; ++k) A.a[k] = k < L->buf.narr ? L->buf.f[copy][k] : nullptr;
    A.st = L->buf.st;
    A.partials = L->buf.partials;
    A.counter = L->buf.counter;
    A.mc = L->mc;
    return A;
}

void su2_geometry(Lattice* L) {
    Geometry& g = L->geo;
    g.N = L->mc.N;
    g.threads = 256;
    const size_t n3 = (size_t)g.N * g.N * g.N;
    int per_sm = 1;
    const bool ext = L->mc.ext != 0;
    if (L->prec == CL_FP32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ext ? su2_kick_kernel<float, true> : su2_kick_kernel<float, false>,
                                                      256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, ext ? su2_kick_kernel<double, true> : su2_kick_kernel<double, false>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)L->sm_count * per_sm;
    const long long need = (long long)((n3 + 255) / 256);
    if (grid > need) grid = need;
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    g.grid = (int)grid;
    g.ntiles = g.grid;
    g.smem = 0;
}

cudaError_t su2_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s) {
    Su2Args S = su2_args(L, src), D = su2_args(L, dst);
    D.pi = pi;
    D.write = write ? 1 : 0;
    const int dg = L->sm_count * 8;
    const int grid = L->geo.grid;
    if (L->mc.ext) {
        if (L->prec == CL_FP32) {
            su2_drift_kernel<float, true><<<dg, 256, 0, s>>>(S, D);
            su2_kick_kernel<float, true><<<grid, 256, 0, s>>>(D);
        } else {
            su2_drift_kernel<double, true><<<dg, 256, 0, s>>>(S, D);
            su2_kick_kernel<double, true><<<grid, 256, 0, s>>>(D);
        }
    } else if (L->prec == CL_FP32) {
        su2_drift_kernel<float, false><<<dg, 256, 0, s>>>(S, D);
        su2_kick_kernel<float, false><<<grid, 256, 0, s>>>(D);
    } else {
        su2_drift_kernel<double, false><<<dg, 256, 0, s>>>(S, D);
        su2_kick_kernel<double, false><<<grid, 256, 0, s>>>(D);
    }
    return cudaGetLastError();
}

cudaError_t su2_launch_drift(Lattice* L, int cur, cudaStream_t s) {
    Su2Args S = su2_args(L, cur);
    const int dg = L->sm_count * 8;
    if (L->mc.ext) {
        if (L->prec == CL_FP32) su2_drift_kernel<float, true><<<dg, 256, 0, s>>>(S, S);
        else su2_drift_kernel<double, true><<<dg, 256, 0, s>>>(S, S);
    } else if (L->prec == CL_FP32) {
        su2_drift_kernel<float, false><<<dg, 256, 0, s>>>(S, S);
    } else {
        su2_drift_kernel<double, false><<<dg, 256, 0, s>>>(S, S);
    }
    return cudaGetLastError();
}

cudaError_t su2_launch_gauss(Lattice* L, int cur, cudaStream_t s) {
    Su2Args A = su2_args(L, cur);
    zero_su2_gauss_kernel<<<1, 1, 0, s>>>(L->buf.st);
    const int grid = L->sm_count * 4;
    if (L->mc.ext) {
        if (L->prec == CL_FP32) su2_gauss_kernel<float, true><<<grid, 256, 0, s>>>(A);
        else su2_gauss_kernel<double, true><<<grid, 256, 0, s>>>(A);
    } else if (L->prec == CL_FP32) {
        su2_gauss_kernel<float, false><<<grid, 256, 0, s>>>(A);
    } else {
        su2_gauss_kernel<double, false><<<grid, 256, 0, s>>>(A);
    }
    return cudaGetLastError();
}

cudaError_t su2_fill(Lattice* L, const double* f, const double* p) {
    Su2Args A = su2_args(L, L->cur);
    const int grid = L->sm_count * 4;
    const int narr = L->buf.narr;
    if (L->prec == CL_FP32)
        su2_fill_kernel<float><<<grid, 256, 0, L->stream>>>(A, narr, f[0], f[1], f[2], f[3], p[0], p[1], p[2], p[3]);
    else
        su2_fill_kernel<double><<<grid, 256, 0, L->stream>>>(A, narr, f[0], f[1], f[2], f[3], p[0], p[1], p[2], p[3]);
    return cudaGetLastError();
}

}  // namespace cl
