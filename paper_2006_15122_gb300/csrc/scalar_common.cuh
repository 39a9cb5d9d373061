// Device functions shared by the single-lattice and the ensemble scalar passes:
// the potential of section 8.1 written as a polynomial in the fluctuation, and
// the FP64 background update that the last block of a pass performs.
#pragma once

#include <math.h>

#include "cl_internal.cuh"

namespace cl {

template <typename T, int P> struct Power;
// (lam/p)|phi|^p: lam * [(fb+d)^{p-1} - fb^{p-1}] and (1/p)[(fb+d)^p - fb^p] as polynomials in d
template <typename T> struct Power<T, 2> {
    static __device__ __forceinline__ T dforce(T fb, T d) { return d; }
    static __device__ __forceinline__ T dvalue(T fb, T d) { return d * (fb + T(0.5) * d); }
};
template <typename T> struct Power<T, 4> {
    static __device__ __forceinline__ T dforce(T fb, T d) { return d * (T(3) * fb * fb + d * (T(3) * fb + d)); }
    static __device__ __forceinline__ T dvalue(T fb, T d) {
        return T(0.25) * d * (T(4) * fb * fb * fb + d * (T(6) * fb * fb + d * (T(4) * fb + d)));
    }
};
template <typename T> struct Power<T, 6> {
    static __device__ __forceinline__ T dforce(T fb, T d) {
        const T f2 = fb * fb;
        return d * (T(5) * f2 * f2 + d * (T(10) * f2 * fb + d * (T(10) * f2 + d * (T(5) * fb + d))));
    }
    static __device__ __forceinline__ T dvalue(T fb, T d) {
        const T f2 = fb * fb;
        return d * (f2 * f2 * fb + d * (T(2.5) * f2 * f2 + d * (T(10.0 / 3.0) * f2 * fb +
                                                              d * (T(2.5) * f2 + d * (fb + d * T(1.0 / 6.0))))));
    }
};

// ------------------------------------------------------------------ finish


static __device__ void potential_bar(const ModelConst& mc, const double* fb, double* V1, double* V2, double* dV) {
    const double f0 = fb[0], f1 = mc.nf > 1 ? fb[1] : 0.0;
    double ap = 1.0;
    for (int i = 0; i < mc.pexp - 2; ++i) ap *= fabs(f0);
    *V1 = mc.lam / mc.pexp * ap * f0 * f0;
    *V2 = mc.nf > 1 ? 0.5 * mc.q * f0 * f0 * f1 * f1 : 0.0;
    dV[0] = mc.lam * ap * f0 + (mc.nf > 1 ? mc.q * f1 * f1 * f0 : 0.0);
    dV[1] = mc.nf > 1 ? mc.q * f0 * f0 * f1 : 0.0;
}

static __device__ double Ka_of(const ModelConst& mc, double a, double EK, double EG, double EV) {
    return mc.fmp2_3 * apow(a, 1.0 + 2.0 * mc.alpha) *
           ((mc.alpha - 2.0) * EK + mc.alpha * EG + (mc.alpha + 1.0) * EV);
}

static __device__ double hubble_rhs(const ModelConst& mc, double a, double Etot) {
    return mc.fmp2_3 * apow(a, 2.0 * (mc.alpha + 1.0)) * Etot;
}

// a^{1+alpha}, a^{3+alpha}, a^{alpha-1}: non-negative powers of a or of 1/a
static __device__ void set_kick_powers(DevState* st, const ModelConst& mc, double a) {
    const double ia = 1.0 / a;
    auto pw = [&](double e) { return e >= 0.0 ? apow(a, e) : apow(ia, -e); };
    st->A1 = pw(1.0 + mc.alpha);
    st->A3 = pw(3.0 + mc.alpha);
    st->Am = pw(mc.alpha - 1.0);
}

// Scalar update of the last block (thread 0).  tot[] are sums / N^3.
static __device__ void scalar_finish(DevState* st, const double* tot, const ModelConst& mc, const PassInfo& pi, bool single) {
    if (st->error) return;
    const int nf = mc.nf;
    const double a = st->a;
    double V1, V2, dV[2];
    potential_bar(mc, st->phibar, &V1, &V2, dV);
    double Kbar[2] = {0, 0}, EK[2] = {0, 0}, EG[2] = {0, 0}, S = 0;
    const double ia = 1.0 / a, ia2 = ia * ia, ia6 = ia2 * ia2 * ia2;
    for (int f = 0; f < nf; ++f) {
        Kbar[f] = -st->A3 * dV[f];
        const double pr = st->pibar[f] + pi.h1 * Kbar[f];
        const double s2 = pr * pr + 2.0 * pr * tot[6 * f + 2] + tot[6 * f + 3];
        S += s2;
        EK[f] = 0.5 * s2 * ia6;
        EG[f] = 0.5 * tot[6 * f + 4] * mc.idx2 * ia2;
    }
    const double EV1 = V1 + tot[6 * nf], EV2 = V2 + tot[6 * nf + 1];
    const double EKt = EK[0] + EK[1], EGt = EG[0] + EG[1], EVt = EV1 + EV2;
    st->E[0] = EK[0]; st->E[1] = EK[1]; st->E[2] = EG[0]; st->E[3] = EG[1]; st->E[4] = EV1; st->E[5] = EV2;
    for (int s = 0; s < 6 * nf + 2 && s < kMaxSums; ++s) st->sums[s] = tot[s];
    if (!isfinite(EKt + EGt + EVt)) { st->error = CL_ERR_NONFINITE; return; }

    const int kind = pi.kind;
    if (kind == PK_MEASURE) {
        if (mc.bg) {
            st->hc = 0.0;
        } else if (st->staggered) {  // scheme III Hubble constraint at the half step behind the fields
            const double rhs = hubble_rhs(mc, st->ahm, st->EKm + 0.5 * (st->EGm + EGt) + 0.5 * (st->EVm + EVt));
            st->hc = rhs > 0 ? fabs(st->b * st->b - rhs) / rhs : 0.0;
        } else {
            const double rhs = hubble_rhs(mc, a, EKt + EGt + EVt);
            st->hc = rhs > 0 ? fabs(st->b * st->b - rhs) / rhs : 0.0;
        }
        return;
    }
    if (kind == PK_INIT_B) {
        if (mc.bg) st->b = bg_b(mc, st->t);
        else st->b = mc.fmp2 > 0 ? sqrt(fmax(hubble_rhs(mc, a, EKt + EGt + EVt), 0.0)) : 0.0;
        st->hc = 0.0;
        return;
    }
    if (kind == PK_LF_EKM) {  // E_K of the momenta half a step behind
        const double ah6 = apow(st->ahm, 6.0);
        st->EKm = S / (2.0 * ah6);
        return;
    }

    double bsync = st->b;
    double bnext = 0.0, anew = a, ah = a;
    if (kind == PK_VV_FIRST || kind == PK_VV_MID || kind == PK_VV_LAST) {
        if (mc.bg) {
            // prescribed background: a and b follow the program time; the
            // Hubble constraint does not apply (reported as 0)
            st->hc = 0.0;
            st->b = bg_b(mc, st->t);
            if (kind != PK_VV_LAST) {
                anew = bg_a(mc, st->t + pi.wn * pi.dt);
                ah = 0.5 * (a + anew);
            }
        } else {
            if (kind == PK_VV_MID || kind == PK_VV_LAST) {
                bsync = st->bh + 0.5 * pi.wc * pi.dt * Ka_of(mc, a, EKt, EGt, EVt);
                const double rhs = hubble_rhs(mc, a, EKt + EGt + EVt);
                st->hc = rhs > 0 ? fabs(bsync * bsync - rhs) / rhs : 0.0;
            }
            if (kind == PK_VV_LAST) {
                st->b = bsync;
            } else {
                bnext = bsync + 0.5 * pi.wn * pi.dt * Ka_of(mc, a, EKt, EGt, EVt);
                st->bh = bnext;
                anew = a + pi.wn * pi.dt * bnext;
                ah = 0.5 * (a + anew);
            }
        }
    } else if (kind == PK_LF) {
        // Scheme III: b_{+1/2} = b_{-1/2} + dt K_a[a, (E_K(-1/2)+E_K(+1/2))/2, E_G, E_V],
        // E_K(+1/2) = S / (2 a_{+1/2}^6), a_{+1/2} = a + dt b_{+1/2}/2: fixed point.
        if (st->staggered && st->ahm > 0) {
            const double rhs = hubble_rhs(mc, st->ahm, st->EKm + 0.5 * (st->EGm + EGt) + 0.5 * (st->EVm + EVt));
            st->hc = rhs > 0 ? fabs(st->b * st->b - rhs) / rhs : 0.0;
        }
        double bp = st->b;
        for (int it = 0; it < 100; ++it) {
            const double ahh = a + 0.5 * pi.dt * bp;
            const double EKp = S / (2.0 * apow(ahh, 6.0));
            const double bn = st->b + pi.dt * Ka_of(mc, a, 0.5 * (st->EKm + EKp), EGt, EVt);
            const double d = fabs(bn - bp);
            bp = bn;
            if (d <= 1e-17 * fabs(bn) || d == 0.0) break;
        }
        anew = a + pi.dt * bp;
        ah = 0.5 * (a + anew);
        st->EKm = S / (2.0 * apow(ah, 6.0));
        st->b = bp;
        st->ahm = ah;
        st->EGm = EGt;
        st->EVm = EVt;
    } else if (kind == PK_LF_PREPARE) {
        const double bm = st->b - 0.5 * pi.dt * Ka_of(mc, a, EKt, EGt, EVt);
        st->b = bm;
        st->ahm = a - 0.5 * pi.dt * bm;
        st->EGm = EGt;
        st->EVm = EVt;
        st->staggered = 1;
    }
    // kick of the means, then move the fluctuations' volume mean into them; the
    // shift is rounded to the arrays' precision so that the FP64 means receive
    // exactly what the arrays give up on their next read
    for (int f = 0; f < nf; ++f) {
        st->pibar[f] += pi.h * Kbar[f];
        double sf = tot[6 * f + 0], sp = tot[6 * f + 5];
        if (single) { sf = (double)(float)sf; sp = (double)(float)sp; }
        st->sphi[f] = sf;
        st->spi[f] = sp;
        st->phibar[f] += sf;
        st->pibar[f] += sp;
    }
    // prepare the drift of the next pass
    double cd = 0.0, dtn = 0.0;
    if (kind == PK_VV_FIRST || kind == PK_VV_MID || kind == PK_LF) {
        dtn = kind == PK_LF ? pi.dt : pi.wn * pi.dt;
        const double iah = 1.0 / ah, e = 3.0 - mc.alpha;
        cd = dtn * (e >= 0.0 ? apow(iah, e) : apow(ah, -e));
    }
    st->cd = cd;
    if (cd != 0.0) {
        for (int f = 0; f < nf; ++f) st->phibar[f] += cd * st->pibar[f];
        st->a = anew;
        set_kick_powers(st, mc, anew);
        st->t += dtn;
    }
}


}  // namespace cl
