// Initial conditions of section 7 on the device.
//
// Scalar singlets (section 7.1): per Fourier mode n~ of the paper's DFT,
//   |dphi(n~)|^2 = (w*/f*)^2 (N/dx)^3 / (2 a^2 w_k),  w_k = sqrt(k^2 + a^2 m^2),
//   dphi(n~)  = (|l| e^{i th_l} + |r| e^{i th_r})/sqrt(2),
//   dphi'(n~) = a^{alpha-1} (i w_k/sqrt(2)) (|l| e^{i th_l} - |r| e^{i th_r}) - H dphi(n~),
// Rayleigh moduli with that mean square, uniform phases.  The half space
// n~_x >= 0 is drawn (cuFFT's R2C layout); modes with n~_x in {0, N/2} are
// paired with their conjugates explicitly, self-conjugate modes take
// sqrt(2) Re, the zero mode is empty, a tachyonic m^2 enters as |m^2|.  The
// draws come from Philox4x32-10 with key = seed and counter = (index of the
// drawing mode in the half layout, stream, draw, 0), so a mode and its
// conjugate share one draw.  The paper's inverse transform
// f(n) = N^-3 sum exp(-2 pi i n~.n/N) f(n~) is cuFFT's C2R (exponent +) fed
// with conj(f(n~)).
//
// Charged scalar with U(1) (section 7.2): the two real components of
// phi = (phi_0 + i phi_1)/sqrt(2) use |l_n| = |r_n| and
// th_1r = th_0r + th_1l - th_0l, so that the total charge vanishes.  The
// doublet of SU(2) x U(1) + chi does the same for its four components
// (th_c^r = th_0^r + th_c^l - th_0^l; moduli from counter (mode, 0, 0), th_0^l,
// th_0^r, th_1^l, th_2^l from (mode, 0, 1), th_3^l from (mode, 0, 2)) with one
// frequency for all of them, which zeroes the U(1) and the three SU(2)
// charges mode by mode.  The links
// start at unity and the electric momenta solve the lattice Gauss law
// sum_i D_i^- piA_i = (2e/kappa) Im[phi* pi] in Fourier space with the
// backward lattice momentum (forward exponent -: gamma_i = (1 - e^{-2 pi i k_i/N})/dx).
#include <math.h>

#include "cl_internal.cuh"

namespace cl {

struct ICParams {
    int N;
    int stream;   // Philox stream (field index)
    int which;    // 0: field, 1: program-time derivative
    int u1comp;   // -1 scalar singlet; else the component of the charged scalar (0/1) or doublet (0..3)
    int doublet;  // the doublet's constrained draws (SU(2) x U(1) + chi)
    double kIR, a, alpha, H;
    double T0;    // (w*/f*)^2 (N/dx)^3 / (2 a^2) * fluct_scale^2
    double m2;    // |m^2| of this component
    uint32_t k0, k1;
};

__device__ __forceinline__ int signed_mode(int i, int N) { return i <= N / 2 ? i : i - N; }
__device__ __forceinline__ int sign_class(int m, int N) { return (m == 0 || m == N / 2) ? 0 : (m > 0 ? 1 : -1); }

__device__ __forceinline__ double u01(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

__global__ void ic_modes_kernel(double2* X, ICParams P) {
    const int N = P.N, NH = N / 2 + 1;
    const size_t total = (size_t)N * N * NH;
    const double r2 = 1.4142135623730951;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % NH);
        const int iy = (int)((i / NH) % N);
        const int iz = (int)(i / ((size_t)NH * N));
        const int mx = ix, my = signed_mode(iy, N), mz = signed_mode(iz, N);
        const int sx = sign_class(mx, N), sy = sign_class(my, N), sz = sign_class(mz, N);
        const bool canon = sx > 0 || (sx == 0 && sy > 0) || (sx == 0 && sy == 0 && sz > 0);
        const bool selfc = sx == 0 && sy == 0 && sz == 0;
        const bool conj = !canon && !selfc;
        if (mx == 0 && my == 0 && mz == 0) { X[i] = make_double2(0.0, 0.0); continue; }
        const int siy = conj ? (N - iy) % N : iy;
        const int siz = conj ? (N - iz) % N : iz;
        const unsigned long long lin = ((unsigned long long)siz * N + siy) * NH + ix;
        const double k = P.kIR * sqrt((double)mx * mx + (double)my * my + (double)mz * mz);
        const double w = sqrt(k * k + P.a * P.a * P.m2);
        const double T = P.T0 / w;
        uint32_t c[4] = {(uint32_t)(lin & 0xffffffffu), (uint32_t)(lin >> 32), (uint32_t)(P.u1comp < 0 ? P.stream : 0), 0u};
        philox4x32_10(c, P.k0, P.k1);
        double L, R, thl, thr;
        if (P.u1comp < 0) {
            L = sqrt(-T * log(u01(c[0])));
            R = sqrt(-T * log(u01(c[1])));
            thl = 2.0 * M_PI * u01(c[2]);
            thr = 2.0 * M_PI * u01(c[3]);
        } else if (P.doublet) {
            // |l_c| = |r_c|; th_c^r = th_0^r + th_c^l - th_0^l
            uint32_t d[4] = {(uint32_t)(lin & 0xffffffffu), (uint32_t)(lin >> 32), 0u, 1u};
            uint32_t e[4] = {(uint32_t)(lin & 0xffffffffu), (uint32_t)(lin >> 32), 0u, 2u};
            philox4x32_10(d, P.k0, P.k1);
            philox4x32_10(e, P.k0, P.k1);
            const double th0l = 2.0 * M_PI * u01(d[0]), th0r = 2.0 * M_PI * u01(d[1]);
            const int cc = P.u1comp;
            const double tl = cc == 0 ? th0l : 2.0 * M_PI * u01(cc == 1 ? d[2] : (cc == 2 ? d[3] : e[0]));
            L = R = sqrt(-T * log(u01(c[cc])));
            thl = tl;
            thr = th0r + tl - th0l;
        } else {
            // |l_n| = |r_n|; th_1r = th_0r + th_1l - th_0l
            uint32_t d[4] = {(uint32_t)(lin & 0xffffffffu), (uint32_t)(lin >> 32), 0u, 1u};
            philox4x32_10(d, P.k0, P.k1);
            const double th0l = 2.0 * M_PI * u01(c[2]), th0r = 2.0 * M_PI * u01(c[3]);
            const double th1l = 2.0 * M_PI * u01(d[0]);
            L = R = sqrt(-T * log(u01(P.u1comp == 0 ? c[0] : c[1])));
            thl = P.u1comp == 0 ? th0l : th1l;
            thr = P.u1comp == 0 ? th0r : th0r + th1l - th0l;
        }
        double sl, cl_, sr, cr;
        sincos(thl, &sl, &cl_);
        sincos(thr, &sr, &cr);
        double gr = (L * cl_ + R * cr) / r2, gi = (L * sl + R * sr) / r2;
        if (P.which == 1) {
            const double dr = L * cl_ - R * cr, di = L * sl - R * sr;
            const double s = pow(P.a, P.alpha - 1.0) * w / r2;
            const double nr = -s * di - P.H * gr, ni = s * dr - P.H * gi;
            gr = nr;
            gi = ni;
        }
        double fr = gr, fi = conj ? -gi : gi;
        if (selfc) { fr = r2 * gr; fi = 0.0; }
        X[i] = make_double2(fr, -fi);  // cuFFT's C2R input is conj(f(n~))
    }
}

template <typename T>
__global__ void store_real_kernel(const double* src, T* dst, size_t n, double scale) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = T(src[i] * scale);
}

// U(1): phi = (phi_0 + i phi_1)/sqrt(2) from the two component arrays (already /N^3 scaled):
// mode 0 writes Re, mode 1 writes Im, with the homogeneous component added.
template <typename T>
__global__ void store_u1_kernel(const double* src, T* dst, size_t n, double scale, double add) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = T((src[i] * scale + add) * 0.70710678118654752);
}

// SU(2): Im[Phi^dag sigma^a pi] of the stored doublet components (a = 0..2)
template <typename T>
__device__ __forceinline__ double su2_rho(const T* const* b, size_t i, int a) {
    const double f0 = b[0][i], f1 = b[1][i], f2 = b[2][i], f3 = b[3][i];
    const double p0 = b[4][i], p1 = b[5][i], p2 = b[6][i], p3 = b[7][i];
    if (a == 0) return f0 * p3 - f1 * p2 + f2 * p1 - f3 * p0;
    if (a == 1) return -f0 * p2 - f1 * p3 + f2 * p0 + f3 * p1;
    return f0 * p1 - f1 * p0 - f2 * p3 + f3 * p2;
}

struct Su2Ptrs {
    void* b[8];  // Phi 0-3, pi 4-7
};

// per-block partial sums of the three colour charges and of |Phi|^2
template <typename T>
__global__ void su2_charge_sums_kernel(const Su2Ptrs P, size_t n, double* partials) {
    const T* const* b = reinterpret_cast<const T* const*>(P.b);
    double s[4] = {0, 0, 0, 0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) s[a] += su2_rho(b, i, a);
        for (int c = 0; c < 4; ++c) s[3] += (double)b[c][i] * (double)b[c][i];
    }
    __shared__ double red[8][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
        const double v = warp_sum(s[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
    }
}

// pi <- pi - sum_a c_a i sigma^a Phi with c_a = Q_a / sum |Phi|^2 (fixed-order sum of the partials)
template <typename T>
__global__ void su2_uncharge_kernel(Su2Ptrs P, size_t n, const double* partials, int nblocks) {
    T* const* b = reinterpret_cast<T* const*>(P.b);
    double q[4] = {0, 0, 0, 0};
    for (int k = 0; k < nblocks; ++k)
        for (int j = 0; j < 4; ++j) q[j] += partials[(size_t)k * 4 + j];
    const double c0 = q[0] / q[3], c1 = q[1] / q[3], c2 = q[2] / q[3];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double f0 = b[0][i], f1 = b[1][i], f2 = b[2][i], f3 = b[3][i];
        // i s1 Phi = (-f3, f2, -f1, f0), i s2 Phi = (f2, f3, -f0, -f1), i s3 Phi = (-f1, f0, f3, -f2)
        b[4][i] = T((double)b[4][i] - (c0 * -f3 + c1 * f2 + c2 * -f1));
        b[5][i] = T((double)b[5][i] - (c0 * f2 + c1 * f3 + c2 * f0));
        b[6][i] = T((double)b[6][i] - (c0 * -f1 + c1 * -f0 + c2 * f3));
        b[7][i] = T((double)b[7][i] - (c0 * f0 + c1 * -f1 + c2 * -f2));
    }
}

// (2 eA/kappa) Im[Phi^dag pi] of the doublet into a real FP64 array
template <typename T>
__global__ void su2_u1_charge_kernel(const Su2Ptrs P, double* rho, size_t n, double c) {
    const T* const* b = reinterpret_cast<const T* const*>(P.b);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double f0 = b[0][i], f1 = b[1][i], f2 = b[2][i], f3 = b[3][i];
        const double p0 = b[4][i], p1 = b[5][i], p2 = b[6][i], p3 = b[7][i];
        rho[i] = c * (f0 * p1 - f1 * p0 + f2 * p3 - f3 * p2);
    }
}

// (g/kappa) Im[Phi^dag sigma^a pi] into a real FP64 array
template <typename T>
__global__ void su2_charge_kernel(const Su2Ptrs P, double* rho, size_t n, int a, double c) {
    const T* const* b = reinterpret_cast<const T* const*>(P.b);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        rho[i] = c * su2_rho(b, i, a);
}

// charge density (2e/kappa) Im[phi* pi] into a real FP64 array
template <typename T>
__global__ void u1_charge_kernel(const T* pr, const T* pim, const T* qr, const T* qi, double* rho, size_t n, double c) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        rho[i] = c * ((double)pr[i] * (double)qi[i] - (double)pim[i] * (double)qr[i]);
}

// Gauss law in Fourier space (forward exponent -): piA_i(k) = conj(g_i) R(k) / sum_j |g_j|^2,
// g_j = (1 - e^{-2 pi i k_j/N})/dx; writes component `comp` into Y (scaled by 1/N^3 for the C2R).
__global__ void u1_gauss_solve_kernel(const double2* R, double2* Y, int N, double dx, int comp) {
    const int NH = N / 2 + 1;
    const size_t total = (size_t)N * N * NH;
    const double invN3 = 1.0 / ((double)N * N * N);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % NH);
        const int iy = (int)((i / NH) % N);
        const int iz = (int)(i / ((size_t)NH * N));
        const int m[3] = {ix, iy, iz};
        double gr[3], gi[3], den = 0.0;
        for (int j = 0; j < 3; ++j) {
            double s, c;
            sincospi(2.0 * m[j] / N, &s, &c);
            gr[j] = (1.0 - c) / dx;  // 1 - e^{-i x} = (1 - cos x) + i sin x
            gi[j] = s / dx;
            den += gr[j] * gr[j] + gi[j] * gi[j];
        }
        const double2 r = R[i];
        if (den <= 0.0) { Y[i] = make_double2(0.0, 0.0); continue; }
        // conj(g) * r
        const double yr = (gr[comp] * r.x + gi[comp] * r.y) / den;
        const double yi = (gr[comp] * r.y - gi[comp] * r.x) / den;
        Y[i] = make_double2(yr * invN3, yi * invN3);
    }
}

static double vbar_scalar(const ModelConst& mc, const double* fb, double* m2) {
    const double f0 = fb[0], f1 = mc.nf > 1 ? fb[1] : 0.0;
    double ap = 1.0;
    for (int i = 0; i < mc.pexp - 2; ++i) ap *= fabs(f0);
    m2[0] = (mc.pexp - 1) * mc.lam * ap + (mc.nf > 1 ? mc.q * f1 * f1 : 0.0);
    m2[1] = mc.nf > 1 ? mc.q * f0 * f0 : 0.0;
    return mc.lam / mc.pexp * ap * f0 * f0 + (mc.nf > 1 ? 0.5 * mc.q * f0 * f0 * f1 * f1 : 0.0);
}

static cudaError_t z2d(Lattice* L) {
    return cufftExecZ2D(L->plan_c2r, (cufftDoubleComplex*)L->cwork, L->work) == CUFFT_SUCCESS ? cudaSuccess
                                                                                                 : cudaErrorUnknown;
}

cl_status ic_generate(Lattice* L) {
    const ModelConst& mc = L->mc;
    const cl_init& in = L->init;
    const int N = mc.N;
    const size_t n = (size_t)N * N * N;
    const double a = in.a0 > 0 ? in.a0 : 1.0;
    const double dx = mc.dx;
    // mc.kappa holds (w*/f*)^2, the amplitude factor of the vacuum fluctuations
    const double base = mc.kappa * pow((double)N / dx, 3.0) / (2.0 * a * a) * in.fluct_scale * in.fluct_scale;
    const int grid = L->sm_count * 8;
    cudaStream_t s = L->stream;
    DevState st;
    memset(&st, 0, sizeof(st));
    st.a = a;
    st.A1 = pow(a, 1.0 + mc.alpha);
    st.A3 = pow(a, 3.0 + mc.alpha);
    st.Am = pow(a, mc.alpha - 1.0);
    if (mc.kind == CL_MODEL_SCALAR) {
        double m2[2];
        const double Vb = vbar_scalar(mc, in.phi0, m2);
        double EK0 = 0.0;
        for (int f = 0; f < mc.nf; ++f) EK0 += in.dphi0[f] * in.dphi0[f];
        EK0 /= 2.0 * pow(a, 2.0 * mc.alpha);
        const double H = sqrt(fmax(pow(a, 2.0 * mc.alpha) / 3.0 * mc.fmp2 * (EK0 + Vb), 0.0));
        for (int f = 0; f < mc.nf; ++f) {
            st.phibar[f] = in.phi0[f];
            st.pibar[f] = pow(a, 3.0 - mc.alpha) * in.dphi0[f];
            for (int which = 0; which < 2; ++which) {
                void* dst = L->buf.f[L->cur][which == 0 ? f : mc.nf + f];
                if (!in.spectrum) {
                    if (cudaMemsetAsync(dst, 0, n * L->tsize, s) != cudaSuccess) return CL_ERR_CUDA;
                    continue;
                }
                ICParams P{};
                P.N = N; P.stream = f; P.which = which; P.u1comp = -1;
                P.kIR = L->grid.kIR; P.a = a; P.alpha = mc.alpha; P.H = H;
                P.T0 = base; P.m2 = fabs(m2[f]);
                P.k0 = (uint32_t)(in.seed & 0xffffffffu); P.k1 = (uint32_t)(in.seed >> 32);
                ic_modes_kernel<<<grid, 256, 0, s>>>((double2*)L->cwork, P);
                if (z2d(L) != cudaSuccess) return CL_ERR_CUDA;
                const double scale = (which == 0 ? 1.0 : pow(a, 3.0 - mc.alpha)) / (double)n;
                if (L->prec == CL_FP32) store_real_kernel<float><<<grid, 256, 0, s>>>(L->work, (float*)dst, n, scale);
                else store_real_kernel<double><<<grid, 256, 0, s>>>(L->work, (double*)dst, n, scale);
            }
        }
    } else if (mc.kind == CL_MODEL_SU2) {
        // SU(2): the homogeneous doublet (stored components), unit links, zero
        // electric field; with a spectrum, every canonical component sqrt(2) Phi_c
        // draws the singlet vacuum fluctuations of its curvature (stream c), the
        // total colour charges are projected out of pi along i sigma^a Phi and the
        // electric momenta solve the unit-link Gauss law colour by colour
        double pb[4];
        for (int c = 0; c < 4; ++c) pb[c] = pow(a, 3.0 - mc.alpha) * in.dphi0[c];
        if (su2_fill(L, in.phi0, pb) != cudaSuccess) return CL_ERR_CUDA;
        if (in.spectrum) {
            double s2 = 0.0, EK0 = 0.0;
            for (int c = 0; c < 4; ++c) {
                s2 += in.phi0[c] * in.phi0[c];
                EK0 += in.dphi0[c] * in.dphi0[c];
            }
            EK0 /= pow(a, 2.0 * mc.alpha);
            double dvb;
            const double Vb = gauge_pot<double>(mc.gpot, mc.pexp, mc.lam, mc.vev2, s2, &dvb);
            const double H = sqrt(fmax(pow(a, 2.0 * mc.alpha) / 3.0 * mc.fmp2 * (EK0 + Vb), 0.0));
            void** b = L->buf.f[L->cur];
            // SU(2) x U(1) + chi: the constrained draws share the mean curvature of the components
            double m2mean = 0.0;
            for (int c = 0; c < 4; ++c)
                m2mean += gauge_curvature(mc.gpot, mc.pexp, mc.lam, mc.vev2, s2, 1.4142135623730951 * in.phi0[c]);
            m2mean /= 4.0;
            for (int c = 0; c < 4; ++c) {
                const double m2 = mc.ext ? m2mean
                                         : gauge_curvature(mc.gpot, mc.pexp, mc.lam, mc.vev2, s2, 1.4142135623730951 * in.phi0[c]);
                for (int which = 0; which < 2; ++which) {
                    ICParams P{};
                    P.N = N; P.stream = c; P.which = which; P.u1comp = mc.ext ? c : -1; P.doublet = mc.ext;
                    P.kIR = L->grid.kIR; P.a = a; P.alpha = mc.alpha; P.H = H;
                    P.T0 = base; P.m2 = fabs(m2);
                    P.k0 = (uint32_t)(in.seed & 0xffffffffu); P.k1 = (uint32_t)(in.seed >> 32);
                    ic_modes_kernel<<<grid, 256, 0, s>>>((double2*)L->cwork, P);
                    if (z2d(L) != cudaSuccess) return CL_ERR_CUDA;
                    const double scale = (which == 0 ? 1.0 : pow(a, 3.0 - mc.alpha)) / (double)n;
                    const double ad = 1.4142135623730951 * (which == 0 ? in.phi0[c] : pow(a, 3.0 - mc.alpha) * in.dphi0[c]);
                    void* dst = b[which == 0 ? c : 4 + c];
                    if (L->prec == CL_FP32) store_u1_kernel<float><<<grid, 256, 0, s>>>(L->work, (float*)dst, n, scale, ad);
                    else store_u1_kernel<double><<<grid, 256, 0, s>>>(L->work, (double*)dst, n, scale, ad);
                }
            }
            if (mc.chi) {  // the singlet: zero mean and velocity, curvature 2 q |Phi|^2, Philox stream 4
                for (int which = 0; which < 2; ++which) {
                    ICParams P{};
                    P.N = N; P.stream = 4; P.which = which; P.u1comp = -1;
                    P.kIR = L->grid.kIR; P.a = a; P.alpha = mc.alpha; P.H = H;
                    P.T0 = base; P.m2 = fabs(2.0 * mc.q * s2);
                    P.k0 = (uint32_t)(in.seed & 0xffffffffu); P.k1 = (uint32_t)(in.seed >> 32);
                    ic_modes_kernel<<<grid, 256, 0, s>>>((double2*)L->cwork, P);
                    if (z2d(L) != cudaSuccess) return CL_ERR_CUDA;
                    const double scale = (which == 0 ? 1.0 : pow(a, 3.0 - mc.alpha)) / (double)n;
                    void* dst = b[35 + which];
                    if (L->prec == CL_FP32) store_real_kernel<float><<<grid, 256, 0, s>>>(L->work, (float*)dst, n, scale);
                    else store_real_kernel<double><<<grid, 256, 0, s>>>(L->work, (double*)dst, n, scale);
                }
            }
            Su2Ptrs P;
            for (int k = 0; k < 8; ++k) P.b[k] = b[k];
            const int cg = L->sm_count * 4;
            if (mc.ext) {
                // no projection: the constrained draws carry no charge
            } else if (L->prec == CL_FP32) {
                su2_charge_sums_kernel<float><<<cg, 256, 0, s>>>(P, n, L->buf.partials);
                su2_uncharge_kernel<float><<<grid, 256, 0, s>>>(P, n, L->buf.partials, cg);
            } else {
                su2_charge_sums_kernel<double><<<cg, 256, 0, s>>>(P, n, L->buf.partials);
                su2_uncharge_kernel<double><<<grid, 256, 0, s>>>(P, n, L->buf.partials, cg);
            }
            double2* Rk = (double2*)L->cwork;
            const size_t nh = (size_t)N * N * (N / 2 + 1);
            double2* Yk = Rk + nh;
            if (mc.e2 > 0) {  // U(1) Gauss law sum_i D_i^- piA_i = (2 eA/kappa) Im[Phi^dag pi]
                if (L->prec == CL_FP32) su2_u1_charge_kernel<float><<<grid, 256, 0, s>>>(P, L->work, n, 2.0 * mc.e2 / mc.kappa);
                else su2_u1_charge_kernel<double><<<grid, 256, 0, s>>>(P, L->work, n, 2.0 * mc.e2 / mc.kappa);
                if (cufftExecD2Z(L->plan_r2c, L->work, (cufftDoubleComplex*)Rk) != CUFFT_SUCCESS) return CL_ERR_CUDA;
                for (int i = 0; i < 3; ++i) {
                    u1_gauss_solve_kernel<<<grid, 256, 0, s>>>(Rk, Yk, N, dx, i);
                    if (cufftExecZ2D(L->plan_c2r, (cufftDoubleComplex*)Yk, L->work) != CUFFT_SUCCESS) return CL_ERR_CUDA;
                    void* dst = b[32 + i];
                    if (L->prec == CL_FP32) store_real_kernel<float><<<grid, 256, 0, s>>>(L->work, (float*)dst, n, 1.0);
                    else store_real_kernel<double><<<grid, 256, 0, s>>>(L->work, (double*)dst, n, 1.0);
                }
            }
            for (int ca = 0; ca < 3; ++ca) {
                if (L->prec == CL_FP32) su2_charge_kernel<float><<<grid, 256, 0, s>>>(P, L->work, n, ca, mc.e / mc.kappa);
                else su2_charge_kernel<double><<<grid, 256, 0, s>>>(P, L->work, n, ca, mc.e / mc.kappa);
                if (cufftExecD2Z(L->plan_r2c, L->work, (cufftDoubleComplex*)Rk) != CUFFT_SUCCESS) return CL_ERR_CUDA;
                for (int i = 0; i < 3; ++i) {
                    u1_gauss_solve_kernel<<<grid, 256, 0, s>>>(Rk, Yk, N, dx, i);
                    if (cufftExecZ2D(L->plan_c2r, (cufftDoubleComplex*)Yk, L->work) != CUFFT_SUCCESS) return CL_ERR_CUDA;
                    void* dst = b[20 + 3 * i + ca];
                    if (L->prec == CL_FP32) store_real_kernel<float><<<grid, 256, 0, s>>>(L->work, (float*)dst, n, 1.0);
                    else store_real_kernel<double><<<grid, 256, 0, s>>>(L->work, (double*)dst, n, 1.0);
                }
            }
        }
    } else {
        // U(1): components phi_0, phi_1 of phi = (phi_0 + i phi_1)/sqrt(2); no mean split
        const double pb[2] = {in.phi0[0], in.phi0[1]}, db[2] = {in.dphi0[0], in.dphi0[1]};
        const double sq = 0.5 * (pb[0] * pb[0] + pb[1] * pb[1]);
        double dvb;
        const double Vb = gauge_pot<double>(mc.gpot, mc.pexp, mc.lam, mc.vev2, sq, &dvb);
        const double EK0 = 0.5 * (db[0] * db[0] + db[1] * db[1]) / pow(a, 2.0 * mc.alpha);
        const double H = sqrt(fmax(pow(a, 2.0 * mc.alpha) / 3.0 * mc.fmp2 * (EK0 + Vb), 0.0));
        for (int comp = 0; comp < 2; ++comp) {
            const double m2 = gauge_curvature(mc.gpot, mc.pexp, mc.lam, mc.vev2, sq, pb[comp]);
            for (int which = 0; which < 2; ++which) {
                void* dst = L->buf.f[L->cur][which == 0 ? comp : 2 + comp];
                const double add = which == 0 ? pb[comp] : db[comp];
                const double scale = (which == 0 ? 1.0 : pow(a, 3.0 - mc.alpha)) / (double)n;
                if (!in.spectrum) {
                    cudaMemsetAsync(L->work, 0, n * sizeof(double), s);
                } else {
                    ICParams P{};
                    P.N = N; P.stream = 0; P.which = which; P.u1comp = comp;
                    P.kIR = L->grid.kIR; P.a = a; P.alpha = mc.alpha; P.H = H;
                    P.T0 = base; P.m2 = fabs(m2);
                    P.k0 = (uint32_t)(in.seed & 0xffffffffu); P.k1 = (uint32_t)(in.seed >> 32);
                    ic_modes_kernel<<<grid, 256, 0, s>>>((double2*)L->cwork, P);
                    if (z2d(L) != cudaSuccess) return CL_ERR_CUDA;
                }
                const double ad = which == 0 ? add : pow(a, 3.0 - mc.alpha) * add;
                if (L->prec == CL_FP32) store_u1_kernel<float><<<grid, 256, 0, s>>>(L->work, (float*)dst, n, scale, ad);
                else store_u1_kernel<double><<<grid, 256, 0, s>>>(L->work, (double*)dst, n, scale, ad);
            }
        }
        // links at unity, electric momenta from the Gauss law
        for (int i = 0; i < 3; ++i)
            if (cudaMemsetAsync(L->buf.f[L->cur][4 + i], 0, n * L->tsize, s) != cudaSuccess) return CL_ERR_CUDA;
        void** b = L->buf.f[L->cur];
        const double c = 2.0 * mc.e / mc.kappa;
        if (L->prec == CL_FP32)
            u1_charge_kernel<float><<<grid, 256, 0, s>>>((const float*)b[0], (const float*)b[1], (const float*)b[2],
                                                         (const float*)b[3], L->work, n, c);
        else
            u1_charge_kernel<double><<<grid, 256, 0, s>>>((const double*)b[0], (const double*)b[1],
                                                          (const double*)b[2], (const double*)b[3], L->work, n, c);
        double2* Rk = (double2*)L->cwork;
        const size_t nh = (size_t)N * N * (N / 2 + 1);
        double2* Yk = Rk + nh;
        if (cufftExecD2Z(L->plan_r2c, L->work, (cufftDoubleComplex*)Rk) != CUFFT_SUCCESS) return CL_ERR_CUDA;
        for (int i = 0; i < 3; ++i) {
            u1_gauss_solve_kernel<<<grid, 256, 0, s>>>(Rk, Yk, N, dx, i);
            if (cufftExecZ2D(L->plan_c2r, (cufftDoubleComplex*)Yk, L->work) != CUFFT_SUCCESS) return CL_ERR_CUDA;
            if (L->prec == CL_FP32) store_real_kernel<float><<<grid, 256, 0, s>>>(L->work, (float*)b[7 + i], n, 1.0);
            else store_real_kernel<double><<<grid, 256, 0, s>>>(L->work, (double*)b[7 + i], n, 1.0);
        }
    }
    if (cudaMemcpyAsync(L->buf.st, &st, sizeof(st), cudaMemcpyHostToDevice, s) != cudaSuccess) return CL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}

__global__ void finish_drift_kernel(DevState* st) {
    for (int f = 0; f < kMaxComp; ++f) st->sphi[f] = 0.0;
    st->cd = 0.0;
    st->cdA = 0.0;
}

cudaError_t launch_finish_drift(Lattice* L, cudaStream_t s) {
    finish_drift_kernel<<<1, 1, 0, s>>>(L->buf.st);
    return cudaGetLastError();
}

}  // namespace cl
