// Compact U(1) sector (paper section 5.3): a complex scalar phi with
// momentum pi = a^{3-alpha} phi' and link angles theta_i = e dx A_i
// (V_i = exp(-i theta_i)) with electric momenta piA_i = a^{1-alpha} F_0i.
//
// Kernels (section 5.3, both derived from one lattice action so that the
// discrete Gauss law holds exactly):
//   K_phi  = -a^{3+alpha} (lam/2)(|phi|^2 - v2) phi
//            + a^{1+alpha} sum_i (V_i phi(n+i) - 2 phi + V_i*(n-i) phi(n-i)) / dx^2
//   K_A,i  = a^{1+alpha} (2e/dx)(1/kappa) Im[phi*(n) V_i(n) phi(n+i)]
//            + a^{alpha-1}/(e dx^3) sum_{j!=i} [Im V_ij(n) - Im V_ij(n-j)],
//   V_ij(n) = V_i(n) V_j(n+i) V_i*(n+j) V_j*(n) = exp(-i theta_ij),
//   theta_ij(n) = theta_i(n) + theta_j(n+i) - theta_i(n+j) - theta_j(n),
// kappa = (w*/f*)^2.  Drifts (compact staggered leapfrog, section 5.3.1, and
// the compact velocity-Verlet VV2..VV10 of sections 5.3.2-5.3.3 with dt -> w_p dt):
//   phi <- phi + dt a_{1/2}^{-(3-alpha)} pi,
//   V_i <- exp(-i e dx dt a_{1/2}^{-(1-alpha)} piA_i) V_i  (theta_i += ..., wrapped to [-pi, pi)),
// the exact exponential of the link drift (unitary for any step).
// Energies (section 5.4.1): E_K^phi = <|pi|^2>/a^6, E_G^phi = sum_i <|D_i^+ phi|^2>/a^2,
// E_V = <V>, E_K^A = kappa/(2a^4) sum_i <piA_i^2>,
// E_G^A = kappa/(a^4 e^2 dx^4) sum_{i<j} <1 - cos theta_ij>.
//
// Each array is read once from HBM (plus halo re-reads, mostly L2 hits) and
// written once per pass; the last block does the FP64 leapfrog/Friedmann
// update as in the scalar pass.
#include <math.h>

#include "cl_internal.cuh"
#include "gauge_finish.cuh"

namespace cl {

struct U1Args {
    const void* in[10];
    void* out[10];
    DevState* st;
    double* partials;
    unsigned int* counter;
    ModelConst mc;
    PassInfo pi;
    int write;
};



template <typename T> __device__ __forceinline__ T wrap_angle(T t) {
    const T twopi = T(6.283185307179586476925287);
    return t - twopi * rint(t / twopi);
}
template <typename T> __device__ __forceinline__ void sc(T x, T* s, T* c);
// FP32: the hardware approximation (the arguments are sums of at most four
// wrapped angles, |x| <= 4 pi); every thread evaluates a shared plaquette from
// the same inputs in the same order, so the cancellations behind the Gauss law
// stay exact
template <> __device__ __forceinline__ void sc<float>(float x, float* s, float* c) { __sincosf(x, s, c); }
template <> __device__ __forceinline__ void sc<double>(double x, double* s, double* c) { sincos(x, s, c); }

// Tile of BX x BY sites marching ZC planes in z (one site per thread).  The
// planes z0-1 .. z0+ZC of all ten arrays, with x/y halos and the two corners
// that the halo plaquettes need, stream through an S-stage shared-memory ring
// (cp.async, one barrier per plane) and are drifted in place.  Every site's
// link phases (cos, sin theta_i) and forward plaquette sines are evaluated
// once, by the thread that owns the site or (for the tile's left column and
// bottom row) by the edge thread that loaded it, and kept in a three-plane
// ring, so 6 sincos per site instead of 15 and each shared plaquette is the
// same number wherever it enters (the Gauss-law cancellation stays exact).
// The kick of plane q runs one iteration after its plaquettes, when the
// neighbours' values are visible.
struct U1TileXY {
    int x0, y0, z0;
};

__device__ __forceinline__ U1TileXY u1_decode_tile(const Geometry& g, int tile) {
    const int tyi = tile % g.nty;
    const int rr = tile / g.nty;
    U1TileXY t;
    t.x0 = (rr % g.ntx) * g.BX;
    t.y0 = tyi * g.BY;
    t.z0 = (rr / g.ntx) * g.ZC;
    return t;
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) u1_pass_kernel(const U1Args A, const Geometry G) {
    DevState* st = A.st;
    if (st->error) return;
    const int N = G.N, BX = G.BX, BY = G.BY, ZC = G.ZC, S = G.S;
    const int RW = BX + 2, ASZ = RW * (BY + 2), STG = 10 * ASZ;  // stage: 10 arrays with halos
    const int PW = BX + 1, PSZ = PW * (BY + 1), SLOT = 9 * PSZ;   // plane of link phases / plaquette sines
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    T* pl = sm + (size_t)S * STG;
    __shared__ double bacc[8][U1NS];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int lin = ty * BX + tx, nthr = BX * BY;
    const int lane = lin & 31, warp = lin >> 5, nwarps = (nthr + 31) >> 5;
    const int nlanes = min(32, nthr - 32 * warp);
    for (int i = lin; i < 8 * U1NS; i += nthr) (&bacc[0][0])[i] = 0.0;

    const T cd = T(st->cd), cdA = T(st->cdA), A1 = T(st->A1), A3 = T(st->A3), Am = T(st->Am);
    const T h1 = T(A.pi.h1), h = T(A.pi.h), idx2 = T(A.mc.idx2);
    const T lam = T(A.mc.lam), v2 = T(A.mc.vev2);
    const T cJ = T(2.0 * A.mc.e / A.mc.dx / A.mc.kappa), cB = T(1.0 / (A.mc.e * A.mc.dx * A.mc.dx * A.mc.dx));
    const size_t NN = (size_t)N * N;

    const int my_tiles = (blockIdx.x < (unsigned)G.ntiles) ? (G.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto wrapN = [&](int v) { return v < 0 ? v + N : (v >= N ? v - N : v); };
    const int oc = (ty + 1) * RW + tx + 1;  // own cell in a stage array
    const int po = (ty + 1) * PW + tx + 1;  // own cell in a plaquette-ring array

    // loader: plane (z0 - 1 + ld_p) of tile ld_k into stage ld_slot; every thread copies its own
    // cell, edge threads the halo cells and the two corners (top-left, bottom-right)
    int ld_k = 0, ld_p = 0, ld_slot = 0;
    U1TileXY ld_t = u1_decode_tile(G, (int)blockIdx.x);
    auto issue = [&]() {
        if (ld_k < my_tiles) {
            const int z = wrapN(ld_t.z0 - 1 + ld_p);
            T* dst = sm + (size_t)ld_slot * STG;
            const int x = ld_t.x0 + tx, y = ld_t.y0 + ty;
            const int xl = wrapN(ld_t.x0 - 1), xr = wrapN(ld_t.x0 + BX), yb = wrapN(ld_t.y0 - 1), yt = wrapN(ld_t.y0 + BY);
#pragma unroll
            for (int a = 0; a < 10; ++a) {
                const T* src = static_cast<const T*>(A.in[a]) + (size_t)z * NN;
                T* d = dst + a * ASZ;
                cp_async_elem(d + oc, src + (size_t)y * N + x);
                if (tx == 0) cp_async_elem(d + (ty + 1) * RW, src + (size_t)y * N + xl);
                if (tx == BX - 1) cp_async_elem(d + (ty + 1) * RW + BX + 1, src + (size_t)y * N + xr);
                if (ty == 0) cp_async_elem(d + tx + 1, src + (size_t)yb * N + x);
                if (ty == BY - 1) cp_async_elem(d + (BY + 1) * RW + tx + 1, src + (size_t)yt * N + x);
                if (tx == 0 && ty == BY - 1) cp_async_elem(d + (BY + 1) * RW, src + (size_t)yt * N + xl);
                if (tx == BX - 1 && ty == 0) cp_async_elem(d + BX + 1, src + (size_t)yb * N + xr);
            }
            if (++ld_p == ZC + 2) {
                ld_p = 0;
                if (++ld_k < my_tiles) ld_t = u1_decode_tile(G, (int)blockIdx.x + ld_k * (int)gridDim.x);
            }
            if (++ld_slot == S) ld_slot = 0;
        }
        cp_async_commit();
    };
    int issued = 0;
    auto wait_for = [&](int need) {
        switch (issued - 1 - need) {
            case 0: cp_async_wait<0>(); break;
            case 1: cp_async_wait<1>(); break;
            case 2: cp_async_wait<2>(); break;
            case 3: cp_async_wait<3>(); break;
            default: cp_async_wait<4>(); break;
        }
        __syncthreads();
    };
    // in-place drift of one cell of a stage: phi += cd pi, theta_d += cdA piA_d
    auto drift_cell = [&](T* sg, int c) {
        sg[c] = sg[c] + cd * sg[2 * ASZ + c];
        sg[ASZ + c] = sg[ASZ + c] + cd * sg[3 * ASZ + c];
#pragma unroll
        for (int d = 0; d < 3; ++d) sg[(4 + d) * ASZ + c] = sg[(4 + d) * ASZ + c] + cdA * sg[(7 + d) * ASZ + c];
    };

    for (int L = 0; L < S; ++L, ++issued) issue();
    int need = 0;  // load index of the next plane to land
    int sb = 0;    // stage slot of the tile's plane -1

    for (int k = 0; k < my_tiles; ++k) {
        const U1TileXY tt = u1_decode_tile(G, (int)blockIdx.x + k * (int)gridDim.x);
        const int x = tt.x0 + tx, y = tt.y0 + ty;
        auto stage = [&](int pz) { int i = sb + pz + 1; i %= S; return sm + (size_t)i * STG; };
        auto slot = [&](int pz) { return pl + (size_t)((pz + 3) % 3) * SLOT; };
        T ts[U1NS];
#pragma unroll
        for (int i = 0; i < U1NS; ++i) ts[i] = T(0);
        T thn[3] = {T(0), T(0), T(0)};   // own drifted theta at plane p+1
        T phm[2] = {T(0), T(0)};         // own drifted phi at plane q-1 of the kick

        for (int p = -2; p <= ZC; ++p) {
            if (p <= ZC - 1) {
                wait_for(need);  // plane p+1 has landed; every earlier write is visible
                ++need;
            } else {
                __syncthreads();
            }
            if (p >= 1) { issue(); ++issued; }  // the stage of plane p-2 is free
            if (p <= ZC - 1) {                 // drift plane p+1: own cell and the halo cells this thread loaded
                T* sg = stage(p + 1);
                drift_cell(sg, oc);
                if (tx == 0) drift_cell(sg, (ty + 1) * RW);
                if (tx == BX - 1) drift_cell(sg, (ty + 1) * RW + BX + 1);
                if (ty == 0) drift_cell(sg, tx + 1);
                if (ty == BY - 1) drift_cell(sg, (BY + 1) * RW + tx + 1);
                if (tx == 0 && ty == BY - 1) drift_cell(sg, (BY + 1) * RW);
                if (tx == BX - 1 && ty == 0) drift_cell(sg, BX + 1);
#pragma unroll
                for (int d = 0; d < 3; ++d) thn[d] = sg[(4 + d) * ASZ + oc];
            }
            if (p >= -1 && p <= ZC - 1) {  // link phases and forward plaquettes of plane p
                const T* Sg = stage(p);
                const T* Sn = stage(p + 1);
                T* P = slot(p);
                const T* G0 = Sg + 4 * ASZ;
                const T* G1 = Sg + 5 * ASZ;
                const T* G2 = Sg + 6 * ASZ;
                const T t0 = G0[oc], t1 = G1[oc], t2 = G2[oc];
                T c, s;
                sc<T>(t0, &s, &c); P[0 * PSZ + po] = c; P[1 * PSZ + po] = s;
                sc<T>(t1, &s, &c); P[2 * PSZ + po] = c; P[3 * PSZ + po] = s;
                sc<T>(t2, &s, &c); P[4 * PSZ + po] = c; P[5 * PSZ + po] = s;
                // theta_ij(n) = theta_i(n) + theta_j(n+i) - theta_i(n+j) - theta_j(n)
                const T q01 = t0 + G1[oc + 1] - G0[oc + RW] - t1;
                const T q02 = t0 + G2[oc + 1] - thn[0] - t2;
                const T q12 = t1 + G2[oc + RW] - thn[1] - t2;
                T c01, c02, c12;
                sc<T>(q01, &s, &c01); P[6 * PSZ + po] = s;
                sc<T>(q02, &s, &c02); P[7 * PSZ + po] = s;
                sc<T>(q12, &s, &c12); P[8 * PSZ + po] = s;
                if (p >= 0) ts[10] += (T(1) - c01) + (T(1) - c02) + (T(1) - c12);
                if (tx == 0) {  // left halo site (x0-1, y): V_0, theta_01, theta_02
                    const int cm = (ty + 1) * RW, pm = (ty + 1) * PW;
                    const T m0 = G0[cm], m1 = G1[cm], m2 = G2[cm];
                    sc<T>(m0, &s, &c); P[0 * PSZ + pm] = c; P[1 * PSZ + pm] = s;
                    sc<T>(m0 + G1[cm + 1] - G0[cm + RW] - m1, &s, &c); P[6 * PSZ + pm] = s;
                    sc<T>(m0 + G2[cm + 1] - Sn[4 * ASZ + cm] - m2, &s, &c); P[7 * PSZ + pm] = s;
                }
                if (ty == 0) {  // bottom halo site (x, y0-1): V_1, theta_01, theta_12
                    const int cm = tx + 1, pm = tx + 1;
                    const T m0 = G0[cm], m1 = G1[cm], m2 = G2[cm];
                    sc<T>(m1, &s, &c); P[2 * PSZ + pm] = c; P[3 * PSZ + pm] = s;
                    sc<T>(m0 + G1[cm + 1] - G0[cm + RW] - m1, &s, &c); P[6 * PSZ + pm] = s;
                    sc<T>(m1 + G2[cm + RW] - Sn[5 * ASZ + cm] - m2, &s, &c); P[8 * PSZ + pm] = s;
                }
            }
            if (p >= 1) {  // kick of plane q = p - 1
                const int q = p - 1;
                const T* Sq = stage(q);
                const T* Su = stage(p);
                const T* P = slot(q);
                const T* Pm = slot(q - 1);
                const T fr = Sq[oc], fi = Sq[ASZ + oc];
                const T pr = Sq[2 * ASZ + oc], pim = Sq[3 * ASZ + oc];
                // neighbours of the site: forward and backward phi, link phases of V_d(n) and V_d(n-d)
                const T fpr[3] = {Sq[oc + 1], Sq[oc + RW], Su[oc]};
                const T fpi[3] = {Sq[ASZ + oc + 1], Sq[ASZ + oc + RW], Su[ASZ + oc]};
                const T fmr[3] = {Sq[oc - 1], Sq[oc - RW], phm[0]};
                const T fmi[3] = {Sq[ASZ + oc - 1], Sq[ASZ + oc - RW], phm[1]};
                const T cm_[3] = {P[0 * PSZ + po - 1], P[2 * PSZ + po - PW], Pm[4 * PSZ + po]};
                const T sm_[3] = {P[1 * PSZ + po - 1], P[3 * PSZ + po - PW], Pm[5 * PSZ + po]};
                T lr = T(-6) * fr, li = T(-6) * fi, grad = T(0), Kj[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const T cc = P[(2 * d) * PSZ + po], s = P[(2 * d + 1) * PSZ + po];
                    // V_d phi(n+d) = (cos t - i sin t)(ur0 + i ui0)
                    const T ur = cc * fpr[d] + s * fpi[d], ui = cc * fpi[d] - s * fpr[d];
                    // V_d*(n-d) phi(n-d) = (cos tm + i sin tm)(wr0 + i wi0)
                    const T wr = cm_[d] * fmr[d] - sm_[d] * fmi[d], wi = cm_[d] * fmi[d] + sm_[d] * fmr[d];
                    lr += ur + wr;
                    li += ui + wi;
                    const T gr = ur - fr, gi = ui - fi;
                    grad += gr * gr + gi * gi;
                    Kj[d] = cJ * (fr * ui - fi * ur);  // (2e/dx)(1/kappa) Im[phi* V_d phi(n+d)]
                }
                // sum_{j != i} [Im V_ij(n) - Im V_ij(n-j)], Im V_ij = -sin(theta_ij), theta_ji = -theta_ij
                const T S01 = P[6 * PSZ + po], S02 = P[7 * PSZ + po], S12 = P[8 * PSZ + po];
                T mag[3];
                mag[0] = (-S01 + P[6 * PSZ + po - PW]) + (-S02 + Pm[7 * PSZ + po]);
                mag[1] = (S01 - P[6 * PSZ + po - 1]) + (-S12 + Pm[8 * PSZ + po]);
                mag[2] = (S02 - P[7 * PSZ + po - 1]) + (S12 - P[8 * PSZ + po - PW]);
                const T mod2 = fr * fr + fi * fi;
                T dv;
                const T vpot = gauge_pot<T>(A.mc.gpot, A.mc.pexp, lam, v2, mod2, &dv);
                const T Kr = -A3 * dv * fr + A1 * lr * idx2, Ki = -A3 * dv * fi + A1 * li * idx2;
                const T prr = pr + h1 * Kr, pri = pim + h1 * Ki;
                const T por = pr + h * Kr, poi = pim + h * Ki;
                T sA = T(0), eo[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const T K = A1 * Kj[d] + Am * cB * mag[d];
                    const T ea = Sq[(7 + d) * ASZ + oc];
                    const T er = ea + h1 * K;
                    eo[d] = ea + h * K;
                    sA += er * er;
                }
                ts[0] += fr; ts[1] += fi; ts[2] += fr * fr; ts[3] += fi * fi;
                ts[4] += prr; ts[5] += pri; ts[6] += prr * prr + pri * pri;
                ts[7] += grad * idx2;
                ts[8] += vpot;
                ts[9] += sA;
                if (A.write) {
                    const size_t o = (size_t)(tt.z0 + q) * NN + (size_t)y * N + x;
                    static_cast<T*>(A.out[0])[o] = fr;
                    static_cast<T*>(A.out[1])[o] = fi;
                    static_cast<T*>(A.out[2])[o] = por;
                    static_cast<T*>(A.out[3])[o] = poi;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        static_cast<T*>(A.out[4 + d])[o] = wrap_angle(Sq[(4 + d) * ASZ + oc]);
                        static_cast<T*>(A.out[7 + d])[o] = eo[d];
                    }
                }
            }
            if (p >= 0) {  // own drifted phi at plane p-1 for the next kick
                const T* Sm = stage(p - 1);
                phm[0] = Sm[oc];
                phm[1] = Sm[ASZ + oc];
            }
        }
        __syncthreads();  // the stages of planes ZC-1 and ZC are free
        issue();
        issue();
        issued += 2;
        sb = (sb + ZC + 2) % S;
#pragma unroll
        for (int i = 0; i < U1NS; ++i) {
            const T v = partial_warp_sum(ts[i], lane, nlanes);
            if (lane == 0) bacc[warp][i] += double(v);
        }
    }
    cp_async_wait<0>();
    __syncthreads();

    // block reduction (FP64), partials, last block
    if (lin < U1NS) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += bacc[w][lin];
        A.partials[(size_t)blockIdx.x * U1NS + lin] = t;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int last;
    if (lin == 0) last = (atomicAdd(A.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[U1NS];
    const double invV = 1.0 / ((double)N * N * N);
    for (int s = warp; s < U1NS; s += nwarps) {
        double ks = 0.0, kc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += nlanes) {
            const double xv = __ldcg(&A.partials[(size_t)b * U1NS + s]);
            const double yk = xv - kc, tk = ks + yk;
            kc = (tk - ks) - yk;
            ks = tk;
        }
        const double r = partial_warp_sum(ks - kc, lane, nlanes);
        if (lane == 0) tot[s] = r * invV;
    }
    __syncthreads();
    if (lin == 0) {
        *A.counter = 0u;
        u1_finish(st, tot, A.mc, A.pi);
    }
}

// Closing drift of the leapfrog (in place): phi += cd pi, theta += cdA piA (wrapped).
template <typename T>
__global__ void u1_drift_kernel(T* pr, T* pim, const T* qr, const T* qi, T* t0, T* t1, T* t2, const T* e0,
                                const T* e1, const T* e2, size_t n, DevState* st) {
    if (st->error) return;
    const T cd = T(st->cd), cdA = T(st->cdA);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        pr[i] += cd * qr[i];
        pim[i] += cd * qi[i];
        t0[i] = wrap_angle(t0[i] + cdA * e0[i]);
        t1[i] = wrap_angle(t1[i] + cdA * e1[i]);
        t2[i] = wrap_angle(t2[i] + cdA * e2[i]);
    }
}

// Gauss-law residual G = sum_i D_i^- piA_i - (2e/kappa) Im[phi* pi] (section 5.2), FP64 sums.
template <typename T>
__global__ void u1_gauss_kernel(const T* pr, const T* pim, const T* qr, const T* qi, const T* e0, const T* e1,
                                const T* e2, int N, double idx, double c, DevState* st) {
    const size_t n3 = (size_t)N * N * N;
    double g2 = 0, l2 = 0, r2 = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
        const size_t mx = ((size_t)z * N + y) * N + (x == 0 ? N - 1 : x - 1);
        const size_t my = ((size_t)z * N + (y == 0 ? N - 1 : y - 1)) * N + x;
        const size_t mz = ((size_t)(z == 0 ? N - 1 : z - 1) * N + y) * N + x;
        const double div = ((double)e0[i] - (double)e0[mx] + (double)e1[i] - (double)e1[my] + (double)e2[i] -
                            (double)e2[mz]) * idx;
        const double rho = c * ((double)pr[i] * (double)qi[i] - (double)pim[i] * (double)qr[i]);
        g2 += (div - rho) * (div - rho);
        l2 += div * div;
        r2 += rho * rho;
    }
    g2 = warp_sum(g2);
    l2 = warp_sum(l2);
    r2 = warp_sum(r2);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st->gauss[0], g2 / (double)n3);
        atomicAdd(&st->gauss[1], l2 / (double)n3);
        atomicAdd(&st->gauss[2], r2 / (double)n3);
    }
}

__global__ void zero_gauss_kernel(DevState* st) { st->gauss[0] = st->gauss[1] = st->gauss[2] = 0.0; }

// Tile geometry of the U(1) pass: BX x BY = 32 x 8 sites (smaller when N is
// smaller), S = 5 stages, and the z-chunk ZC in {128, ..., 8} that best
// balances the tiles over the resident blocks against the two extra planes a
// chunk loads.
void u1_geometry(Lattice* L) {
    Geometry& g = L->geo;
    const int N = L->mc.N;
    g.N = N;
    g.V = 1;
    g.BX = N < 32 ? N : 32;
    g.BY = N < 8 ? N : 8;
    g.S = 5;
    g.threads = g.BX * g.BY;
    g.ntx = N / g.BX;
    g.nty = N / g.BY;
    const size_t ts = L->prec == CL_FP32 ? 4 : 8;
    g.smem = ts * ((size_t)g.S * 10 * (g.BX + 2) * (g.BY + 2) + 3 * 9 * (size_t)(g.BX + 1) * (g.BY + 1));
    const void* fn = L->prec == CL_FP32 ? (const void*)u1_pass_kernel<float> : (const void*)u1_pass_kernel<double>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    cudaGetLastError();
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g.threads, g.smem);
    if (per_sm < 1) per_sm = 1;
    const long long resident = (long long)L->sm_count * per_sm;
    double best = -1.0;
    int zc_best = 8 < N ? 8 : N;
    for (int zc = 128; zc >= 8; zc /= 2) {
        if (zc > N || N % zc != 0) continue;
        const long long nt = (long long)g.ntx * g.nty * (N / zc);
        const long long grid = nt < resident ? nt : resident;
        const long long rounds = (nt + grid - 1) / grid;
        const double eff = (double)nt / (double)(rounds * resident) * zc / (zc + 2.0);
        if (eff > best + 1e-9) { best = eff; zc_best = zc; }
    }
    g.ZC = zc_best;
    g.ntz = N / g.ZC;
    g.ntiles = g.ntx * g.nty * g.ntz;
    long long grid = resident < g.ntiles ? resident : g.ntiles;
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    g.grid = (int)grid;
}

cudaError_t u1_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s) {
    U1Args A;
    for (int i = 0; i < 10; ++i) {
        A.in[i] = L->buf.f[src][i];
        A.out[i] = L->buf.f[dst][i];
    }
    A.st = L->buf.st;
    A.partials = L->buf.partials;
    A.counter = L->buf.counter;
    A.mc = L->mc;
    A.pi = pi;
    A.write = write ? 1 : 0;
    const Geometry& g = L->geo;
    const dim3 block(g.BX, g.BY);
    if (L->prec == CL_FP32) u1_pass_kernel<float><<<g.grid, block, g.smem, s>>>(A, g);
    else u1_pass_kernel<double><<<g.grid, block, g.smem, s>>>(A, g);
    return cudaGetLastError();
}

cudaError_t u1_launch_drift(Lattice* L, int cur, cudaStream_t s) {
    void** b = L->buf.f[cur];
    const size_t n = (size_t)L->mc.N * L->mc.N * L->mc.N;
    const int grid = L->sm_count * 8;
    if (L->prec == CL_FP32)
        u1_drift_kernel<float><<<grid, 256, 0, s>>>((float*)b[0], (float*)b[1], (const float*)b[2], (const float*)b[3],
                                                    (float*)b[4], (float*)b[5], (float*)b[6], (const float*)b[7],
                                                    (const float*)b[8], (const float*)b[9], n, L->buf.st);
    else
        u1_drift_kernel<double><<<grid, 256, 0, s>>>((double*)b[0], (double*)b[1], (const double*)b[2],
                                                     (const double*)b[3], (double*)b[4], (double*)b[5], (double*)b[6],
                                                     (const double*)b[7], (const double*)b[8], (const double*)b[9], n,
                                                     L->buf.st);
    return cudaGetLastError();
}

cudaError_t u1_launch_gauss(Lattice* L, int cur, cudaStream_t s) {
    void** b = L->buf.f[cur];
    zero_gauss_kernel<<<1, 1, 0, s>>>(L->buf.st);
    const int grid = L->sm_count * 4;
    const double c = 2.0 * L->mc.e / L->mc.kappa, idx = 1.0 / L->mc.dx;
    if (L->prec == CL_FP32)
        u1_gauss_kernel<float><<<grid, 256, 0, s>>>((const float*)b[0], (const float*)b[1], (const float*)b[2],
                                                    (const float*)b[3], (const float*)b[7], (const float*)b[8],
                                                    (const float*)b[9], L->mc.N, idx, c, L->buf.st);
    else
        u1_gauss_kernel<double><<<grid, 256, 0, s>>>((const double*)b[0], (const double*)b[1], (const double*)b[2],
                                                     (const double*)b[3], (const double*)b[7], (const double*)b[8],
                                                     (const double*)b[9], L->mc.N, idx, c, L->buf.st);
    return cudaGetLastError();
}

}  // namespace cl
