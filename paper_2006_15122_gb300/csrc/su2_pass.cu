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
// One pass = a drift kernel (fields and links, src copy -> dst copy,
// pointwise) followed by a kick kernel that reads the drifted fields and links
// of dst through a shared-memory plane ring, the momenta of src, and writes
// the kicked momenta to dst; it also reduces the volume sums and runs the FP64
// background update in its last block, shared with the U(1) sector.  Array slots: 0-3 Phi (Re/Im of the two components),
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
#include <stdlib.h>

#include "cl_internal.cuh"
#include "gauge_finish.cuh"
#include "plane_ring.cuh"

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

// ------------------------------------------------------------ tiled kick
//
// The kick reads Phi and the links (and with EXT the U(1) angles and the
// singlet) at the site and its neighbours: n +- i, and for the plaquettes
// n + i + j, n - j + i.  Those arrays go through the shared-memory plane ring
// of plane_ring.cuh (BX x 8 tiles, one site per thread); the momenta are read
// and written at the own site only.

// staged array k -> slot in the 37-array layout: Phi 0-3, links 8-19,
// U(1) angles 29-31, singlet 35
__host__ __device__ constexpr int su2_stage_slot(int k) {
    return k < 4 ? k : (k < 16 ? 8 + (k - 4) : (k < 19 ? 29 + (k - 16) : 35));
}
template <bool EXT> __host__ __device__ constexpr int su2_staged() { return EXT ? 20 : 16; }
constexpr int kSu2TileBY = 8;

template <typename T, bool EXT, int BX>
__global__ void __launch_bounds__(BX * kSu2TileBY, (sizeof(T) == 4 && !EXT ? 512 : 256) / (BX * kSu2TileBY))
    su2_kick_kernel(const Su2Args A, const Su2Args P, const int S) {
    constexpr int NS = EXT ? kSu2ExtNS : U1NS;
    constexpr int BY = kSu2TileBY, NT = BX * BY;
    constexpr int NA = su2_staged<EXT>();
    using Ring = PlaneRing<T, NA, BX, BY>;
    constexpr int V = Ring::V, RW = Ring::RW, ASZ = Ring::ASZ;
    DevState* st = A.st;
    if (st->error) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw + 128);
    __shared__ const T* s_src[NA];
    const int N = A.mc.N;
    T* const* arr = reinterpret_cast<T* const*>(A.a);
    T* const* parr = reinterpret_cast<T* const*>(P.a);  // momenta before the kick (the pass's source copy)
    const int tx = threadIdx.x, ty = threadIdx.y, lin = ty * BX + tx;
    if (lin == 0) {
#pragma unroll
        for (int k = 0; k < NA; ++k) s_src[k] = arr[su2_stage_slot(k)];
    }
    const T A1 = T(st->A1), A3 = T(st->A3), Am = T(st->Am);
    const T h1 = T(A.pi.h1), h = T(A.pi.h), idx2 = T(A.mc.idx2);
    const T lam = T(A.mc.lam), v2 = T(A.mc.vev2);
    const T cJ = T(A.mc.e / (A.mc.kappa * A.mc.dx)), cM = T(2.0 / (A.mc.e * A.mc.dx * A.mc.dx * A.mc.dx));
    const bool hasA = EXT && A.mc.e2 > 0, hasC = EXT && A.mc.chi;
    const T cJA = hasA ? T(2.0 * A.mc.e2 / (A.mc.kappa * A.mc.dx)) : T(0);
    const T cMA = hasA ? T(1.0 / (A.mc.e2 * A.mc.dx * A.mc.dx * A.mc.dx)) : T(0);
    const T qc = T(A.mc.q);
    const size_t n3 = (size_t)N * N * N, NN = (size_t)N * N;

    __syncthreads();  // s_src
    Ring ring;
    ring.start(sm, s_src, N, S, lin);

    // per-thread sums in T, folded into FP64 every 64 sites
    double acc[NS];
    T ts[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) { acc[s] = 0.0; ts[s] = T(0); }
    int cnt = 0;

    const int own = (ty + 1) * RW + V + tx;
    for (long long cur = ring.beg; cur < ring.end;) {
        const typename Ring::Seg sg = ring.seg_at(cur);
        const int x = sg.x0 + tx, y = sg.y0 + ty;
        for (int zz = 0; zz < sg.len; ++zz) {
            ring.begin_plane(zz);  // planes z-1, z, z+1 resident
            const T* bs[3] = {ring.stage(-1) + own, ring.stage(0) + own, ring.stage(1) + own};
            const size_t n = (size_t)(sg.z0 + zz) * NN + (size_t)y * N + x;
            if (zz + 1 < sg.len) {  // the momenta of the next plane into L2
#pragma unroll
                for (int k = 4; k < 8; ++k) prefetch_l2(parr[k] + n + NN);
#pragma unroll
                for (int k = 20; k < 29; ++k) prefetch_l2(parr[k] + n + NN);
                if (hasA) {
#pragma unroll
                    for (int k = 32; k < 35; ++k) prefetch_l2(parr[k] + n + NN);
                }
                if (hasC) prefetch_l2(parr[36] + n + NN);
            }
            // the own momenta, loaded before the compute so their latency hides behind it
            T pm0[4], pe0[9];
#pragma unroll
            for (int c = 0; c < 4; ++c) pm0[c] = __ldcs(parr[4 + c] + n);
#pragma unroll
            for (int k = 0; k < 9; ++k) pe0[k] = __ldcs(parr[20 + k] + n);
            T pa0[3] = {T(0), T(0), T(0)}, pc0 = T(0);
            if (hasA) {
#pragma unroll
                for (int k = 0; k < 3; ++k) pa0[k] = __ldcs(parr[32 + k] + n);
            }
            if (hasC) pc0 = __ldcs(parr[36] + n);
            // staged array a at the neighbour (ox, oy, oz)
            auto at = [&](int a, int ox, int oy, int oz) -> T { return bs[oz + 1][a * ASZ + oy * RW + ox]; };
            auto ldq_s = [&](int i, int ox, int oy, int oz, T* q) {
#pragma unroll
                for (int c = 0; c < 4; ++c) q[c] = at(4 + 4 * i + c, ox, oy, oz);
            };
            auto ldf_s = [&](int ox, int oy, int oz, T* f) {
#pragma unroll
                for (int c = 0; c < 4; ++c) f[c] = at(c, ox, oy, oz);
            };

            T f[4], lap[4], grad = T(0), eB = T(0);
            ldf_s(0, 0, 0, f);
#pragma unroll
            for (int c = 0; c < 4; ++c) lap[c] = T(-6) * f[c];
            T KB[3][3];
            // U(1) sector: forward plaquette angles theta_01, theta_02, theta_12 at n (sines, cosines)
            T KA[3] = {T(0), T(0), T(0)}, eBA = T(0), chi0 = T(0), lchi = T(0), gchi = T(0);
            T psn[3] = {T(0), T(0), T(0)};
            if (hasA) {
#pragma unroll
                for (int pr = 0; pr < 3; ++pr) {
                    const int ii = pr == 2 ? 1 : 0, jj = pr == 0 ? 1 : 2;
                    const T p = at(16 + ii, 0, 0, 0) + at(16 + jj, ii == 0, ii == 1, ii == 2) -
                                at(16 + ii, jj == 0, jj == 1, jj == 2) - at(16 + jj, 0, 0, 0);
                    T cs;
                    phase_sc(p, &psn[pr], &cs);
                    eBA += T(1) - cs;
                }
            }
            if (hasC) chi0 = at(19, 0, 0, 0);
            // forward SU(2) plaquettes U_01, U_02, U_12 at n: vector parts and magnetic energy
            // (U_ji = U_ij^dag, so the plane (j, i) takes the vector part with the sign flipped)
            T Pv[3][3];
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
                const int ii = pr == 2 ? 1 : 0, jj = pr == 0 ? 1 : 2;
                T Ui[4], Ujp[4], Uip[4], Uj[4], t1[4], t2[4], c[4], P[4];
                ldq_s(ii, 0, 0, 0, Ui);
                ldq_s(jj, ii == 0, ii == 1, ii == 2, Ujp);
                ldq_s(ii, jj == 0, jj == 1, jj == 2, Uip);
                ldq_s(jj, 0, 0, 0, Uj);
                qmul(Ui, Ujp, t1);
                qconj(Uip, c);
                qmul(t1, c, t2);
                qconj(Uj, c);
                qmul(t2, c, P);
                eB += T(4) * (T(1) - P[0]);
#pragma unroll
                for (int k = 0; k < 3; ++k) Pv[pr][k] = P[k + 1];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int ex = i == 0, ey = i == 1, ez = i == 2;
                T q[4], qm[4], c[4], fp[4], fm[4], t[4], t2[4];
                ldq_s(i, 0, 0, 0, q);
                ldq_s(i, -ex, -ey, -ez, qm);
                qconj(qm, c);
                ldf_s(ex, ey, ez, fp);
                ldf_s(-ex, -ey, -ez, fm);
                umul(q, fp, t);
                umul(c, fm, t2);
                if (hasA) {  // W_i Phi(n+i) = e^{-i theta_i(n)} U_i Phi(n+i); W_i^dag(n-i) = U^dag e^{+i theta_i(n-i)}
                    T sn, cs;
                    phase_sc(at(16 + i, 0, 0, 0), &sn, &cs);
                    phase_minus(t, sn, cs);
                    phase_sc(at(16 + i, -ex, -ey, -ez), &sn, &cs);
                    phase_plus(t2, sn, cs);
                }
                if (hasC) {
                    const T cp = at(19, ex, ey, ez);
                    lchi += cp + at(19, -ex, -ey, -ez);
                    gchi += (cp - chi0) * (cp - chi0);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    lap[k] += t[k] + t2[k];
                    grad += (t[k] - f[k]) * (t[k] - f[k]);
                }
                T js[3];
                im_sigma(f, t, js);
                // backward staples U_j^dag(n-j) U_ij(n-j) U_j(n-j) = X_j U_i^dag(n) with
                // X_j = U_j^dag(n-j) U_i(n-j) U_j(n-j+i) (the factors U_j^dag(n-j) U_j(n-j) = 1 of
                // the plaquette form cancelled, unit links); the product with U_i^dag(n) is
                // linear, so it is taken once on the sum over j
                T mag[3] = {T(0), T(0), T(0)};
                T Xs[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (j == i) continue;
                    const int fx = j == 0, fy = j == 1, fz = j == 2;
                    const int pr = i + j - 1;  // (0,1) -> 0, (0,2) -> 1, (1,2) -> 2
                    const T sg_ = i < j ? T(1) : T(-1);
                    T Uj[4], Ui[4], Ujp[4], cj[4], s1[4], s2[4];
                    ldq_s(j, -fx, -fy, -fz, Uj);
                    ldq_s(i, -fx, -fy, -fz, Ui);
                    ldq_s(j, ex - fx, ey - fy, ez - fz, Ujp);
                    qconj(Uj, cj);
                    qmul(cj, Ui, s1);
                    qmul(s1, Ujp, s2);
#pragma unroll
                    for (int k = 0; k < 4; ++k) Xs[k] += s2[k];
#pragma unroll
                    for (int k = 0; k < 3; ++k) mag[k] += sg_ * Pv[pr][k];
                }
                {
                    T uic[4], Q[4];
                    qconj(q, uic);
                    qmul(Xs, uic, Q);
#pragma unroll
                    for (int k = 0; k < 3; ++k) mag[k] -= Q[k + 1];
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) KB[i][k] = A1 * cJ * js[k] + Am * cM * mag[k];
                if (hasA) {
                    // sum_{j != i} [sin theta_ij(n-j) - sin theta_ij(n)], theta_ji = -theta_ij
                    T magA = T(0);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        if (j == i) continue;
                        const int fx = j == 0, fy = j == 1, fz = j == 2;
                        const int ii = i < j ? i : j, jj = i < j ? j : i;
                        const T sgn = i < j ? T(1) : T(-1);
                        // theta_ij(n-j) = theta_i(n-j) + theta_j(n-j+i) - theta_i(n) - theta_j(n-j)
                        const T pm = at(16 + i, -fx, -fy, -fz) + at(16 + j, ex - fx, ey - fy, ez - fz) -
                                     at(16 + i, 0, 0, 0) - at(16 + j, -fx, -fy, -fz);
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
                const T p = pm0[c];
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
                    const T e = pe0[3 * i + k];
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
                    const T e = pa0[i];
                    const T es = e + h1 * KA[i];
                    sAA += es * es;
                    if (A.write) arr[32 + i][n] = e + h * KA[i];
                }
                ts[11 % NS] += sAA;
                ts[12 % NS] += eBA;
            }
            if (hasC) {
                const T Kc = -A3 * T(2) * qc * mod2 * chi0 + A1 * (lchi - T(6) * chi0) * idx2;
                const T p = pc0;
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
            ring.end_plane();
        }
        ring.end_segment();
        cur += sg.len;
    }
    ring.finish();
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] += double(ts[s]);

    // block reduction, partials, last block
    __shared__ double red[NT / 32][NS];
    const int lane = lin & 31, warp = lin >> 5, nwarps = NT / 32;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const double v = partial_warp_sum(acc[s], lane, 32);
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
    const double invV = A.mc.inv_vol;
    for (int s = warp; s < NS; s += nwarps) {
        const double r = warp_partials_sum(A.partials, (int)gridDim.x, NS, s, lane, 32);
        if (lane == 0) tot[s] = r * invV;
    }
    __syncthreads();
    if (lin == 0) {
        *A.counter = 0u;
        u1_finish(st, tot, A.mc, A.pi, NS);
    }
}

// Drift with the coefficients prepared by the last pass: phi += cd pi,
// U_i <- exp(-i cdA piB_i.sigma/2) U_i (renormalised).  The momenta are left to
// the kick, which writes them to dst; the ones it does not kick (piA without the
// U(1) sector, pchi without the singlet) are carried over here.
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
        for (int c = 0; c < 4; ++c) dst[c][n] = src[c][n] + cd * src[4 + c][n];
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
        }
        if (EXT) {
            const T cA = S.mc.e2 > 0 ? T(st->cdA * (S.mc.e2 / S.mc.e)) : T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T e = src[32 + i][n];
                dst[29 + i][n] = S.mc.e2 > 0 ? wrap_phase(src[29 + i][n] + cA * e) : src[29 + i][n];
                if (!(S.mc.e2 > 0)) dst[32 + i][n] = e;  // not kicked: carried over
            }
            const T pc = src[36][n];
            dst[35][n] = src[35][n] + cd * pc;
            if (!S.mc.chi) dst[36][n] = pc;
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

template <typename T, bool EXT, int BX> static const void* su2_kick_ptr() {
    return (const void*)su2_kick_kernel<T, EXT, BX>;
}
static const void* su2_kick_fn(const Lattice* L) {
    const bool ext = L->mc.ext != 0;
    if (L->prec == CL_FP32) {
        if (L->geo.BX == 32) return ext ? su2_kick_ptr<float, true, 32>() : su2_kick_ptr<float, false, 32>();
        return ext ? su2_kick_ptr<float, true, 8>() : su2_kick_ptr<float, false, 8>();
    }
    return ext ? su2_kick_ptr<double, true, 8>() : su2_kick_ptr<double, false, 8>();
}

// Tile of the kick: 32 x 8 sites in FP32 when 32 divides N, else 8 x 8 (FP64
// always: its stages are twice as large).  Ring of S = 4 stages (5 if it fits
// twice per SM); grid = blocks resident per SM x SMs, at most one per plane tile.
void su2_geometry(Lattice* L) {
    Geometry& g = L->geo;
    const int N = L->mc.N;
    g.N = N;
    g.V = L->prec == CL_FP32 ? 4 : 2;
    g.BX = (L->prec == CL_FP32 && N % 32 == 0) ? 32 : 8;
    if (const char* env = getenv("CL_SU2_TILE_X"))  // override: 8 forces the 8 x 8 tile
        if (atoi(env) == 8) g.BX = 8;
    g.BY = kSu2TileBY;
    g.threads = g.BX * g.BY;
    g.ntx = N / g.BX;
    g.nty = N / g.BY;
    const int na = L->mc.ext ? su2_staged<true>() : su2_staged<false>();
    const size_t stage = (size_t)na * (g.BY + 2) * (g.BX + 2 * g.V) * L->tsize;
    const void* fn = su2_kick_fn(L);
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    cudaGetLastError();
    g.S = 4;
    g.smem = 128 + g.S * stage;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g.threads, g.smem);
    if (per_sm < 1) per_sm = 1;
    {
        int per5 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per5, fn, g.threads, 128 + 5 * stage) == cudaSuccess &&
            per5 >= per_sm) {
            g.S = 5;
            g.smem = 128 + 5 * stage;
        }
        cudaGetLastError();
    }
    const long long W = (long long)g.ntx * g.nty * N;
    long long grid = (long long)L->sm_count * per_sm;
    if (grid > W) grid = W;
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    g.grid = (int)grid;
    g.ntiles = (int)W;
}

template <typename T, bool EXT>
static void su2_pass_t(Lattice* L, const Su2Args& S, const Su2Args& D, cudaStream_t s) {
    const Geometry& g = L->geo;
    su2_drift_kernel<T, EXT><<<L->sm_count * 8, 256, 0, s>>>(S, D);
    const dim3 blk(g.BX, g.BY);
    if (g.BX == 32) su2_kick_kernel<T, EXT, sizeof(T) == 4 ? 32 : 8><<<g.grid, blk, g.smem, s>>>(D, S, g.S);
    else su2_kick_kernel<T, EXT, 8><<<g.grid, blk, g.smem, s>>>(D, S, g.S);
}

cudaError_t su2_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s) {
    Su2Args S = su2_args(L, src), D = su2_args(L, dst);
    D.pi = pi;
    D.write = write ? 1 : 0;
    if (L->mc.ext) {
        if (L->prec == CL_FP32) su2_pass_t<float, true>(L, S, D, s);
        else su2_pass_t<double, true>(L, S, D, s);
    } else if (L->prec == CL_FP32) {
        su2_pass_t<float, false>(L, S, D, s);
    } else {
        su2_pass_t<double, false>(L, S, D, s);
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
