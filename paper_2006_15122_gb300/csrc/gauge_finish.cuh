// FP64 background update of the gauge sectors (last block of a pass), shared
// by the compact U(1) and the SU(2) passes: both reduce the same 11 volume
// sums -- {<f0>, <f1>, <f0^2>, <f1^2>, <p0>, <p1>, <sum |pi_sync|^2>,
// <sum_i |D_i^+ phi|^2>/dx^2, <V>, <sum piA_sync^2>, magnetic sum M} -- with
// E_K^phi = S_pi/a^6, E_G^phi = S_G/a^2, E_V, E_K^A = kappa S_A/(2 a^4) and
// E_G^A = kappa M/(a^4 e^2 dx^4), where M = sum_{i<j} <1 - cos theta_ij> for U(1)
// (section 5.4.1) and M = 2 sum_{i<j} <2 - Tr U_ij> for SU(2) with e = g
// (section 6.3.1).  K_a carries the gauge energies with weight (alpha - 1).
#pragma once

#include "cl_internal.cuh"

namespace cl {

constexpr int U1NS = 11;

// K_a of the gauge models (fmp2_3 = (f*/m_p)^2 / 3).
static __device__ double Ka_u1(const ModelConst& mc, double a, double EKp, double EGp, double EV, double EKA, double EGA) {
    return mc.fmp2_3 * apow(a, 2.0 * mc.alpha + 1.0) *
           ((mc.alpha - 2.0) * EKp + mc.alpha * EGp + (mc.alpha + 1.0) * EV + (mc.alpha - 1.0) * (EKA + EGA));
}

// x^e from x and 1/x: a non-negative power of whichever of the two makes the
// exponent non-negative (no division).
static __device__ __forceinline__ double apow2(double x, double ix, double e) {
    return e >= 0.0 ? apow(x, e) : apow(ix, -e);
}

// SU(2) x U(1) + chi (ns = 15) adds {<sum piA_sync^2>, <sum_{i<j} (1 - cos theta_ij)>,
// <pchi_sync^2>, <sum_i (D_i^+ chi)^2>/dx^2}; the background update then sees the
// scalar sectors (Phi, chi) and the gauge sectors (SU(2), U(1)) in aggregate,
// which is exact because every energy of one class scales with the same power
// of a (chi's kinetic and gradient energies carry the 1/2 of a real field).
// The state is read once and written once, and powers of a come from 1/a, so
// that the chain of dependent FP64 operations of this one thread stays short.
static __device__ void u1_finish(DevState* st, const double* tot, const ModelConst& mc, const PassInfo& pi,
                                 int ns = U1NS) {
    const double a = st->a, b = st->b, bh = st->bh, t = st->t, ahm = st->ahm;
    const double EKm0 = st->EKm, EKAm0 = st->EKAm, EGm0 = st->EGm, EVm0 = st->EVm, EGAm0 = st->EGAm;
    const int staggered = st->staggered;
    const double ia = 1.0 / a, ia2 = ia * ia, ia4 = ia2 * ia2, ia6 = ia4 * ia2;
    double Sp = tot[6], SA = tot[9], SG = tot[7], SM = tot[10] * mc.inv_e_sq;
    if (ns > U1NS) {
        Sp += 0.5 * tot[13];
        SG += 0.5 * tot[14];
        if (mc.e2 > 0) {
            SA += tot[11];
            SM += tot[12] * mc.inv_e2_sq;
        }
    }
    const double hk = 0.5 * mc.kappa;
    const double EKp = Sp * ia6, EGp = SG * ia2, EV = tot[8];
    const double EKA = hk * SA * ia4, EGA = mc.kappa * SM * ia4 * mc.inv_dx4;
    st->E[0] = EKp; st->E[1] = EGp; st->E[2] = EV; st->E[3] = EKA; st->E[4] = EGA;
    for (int s = 0; s < ns; ++s) st->sums[s] = tot[s];
    const double Et = EKp + EGp + EV + EKA + EGA;
    if (!isfinite(Et)) { st->error = CL_ERR_NONFINITE; return; }
    auto rhs = [&](double aa, double E) { return mc.fmp2_3 * apow(aa, 2.0 * (mc.alpha + 1.0)) * E; };
    auto violation = [&](double bb, double r) { return r > 0 ? fabs(bb * bb - r) / r : 0.0; };
    const int kind = pi.kind;
    if (kind == PK_MEASURE) {
        if (mc.bg) st->hc = 0.0;
        else if (staggered)
            st->hc = violation(b, rhs(ahm, EKm0 + EKAm0 + 0.5 * (EGm0 + EGp) + 0.5 * (EVm0 + EV) + 0.5 * (EGAm0 + EGA)));
        else st->hc = violation(b, rhs(a, Et));
        return;
    }
    if (kind == PK_INIT_B) {
        if (mc.bg) st->b = bg_b(mc, t);
        else st->b = mc.fmp2 > 0 ? sqrt(fmax(rhs(a, Et), 0.0)) : 0.0;
        st->hc = 0.0;
        return;
    }
    if (kind == PK_LF_EKM) {
        const double ih = 1.0 / ahm, ih2 = ih * ih, ih4 = ih2 * ih2;
        st->EKm = Sp * ih4 * ih2;
        st->EKAm = hk * SA * ih4;
        return;
    }
    if (kind == PK_LF_PREPARE) {
        const double bm = b - 0.5 * pi.dt * Ka_u1(mc, a, EKp, EGp, EV, EKA, EGA);
        st->b = bm;
        st->ahm = a - 0.5 * pi.dt * bm;
        st->EGm = EGp; st->EVm = EV; st->EGAm = EGA;
        st->staggered = 1;
        st->cd = 0.0;
        st->cdA = 0.0;
        return;
    }
    // the drift of the next pass (a_{1/2} = ah) and the kick powers at the new a
    auto advance = [&](double h, double an) {
        const double ah = 0.5 * (a + an), iah = 1.0 / ah, ian = 1.0 / an;
        st->cd = h * apow(iah, 3.0 - mc.alpha);
        st->cdA = mc.e * mc.dx * h * apow2(iah, ah, 1.0 - mc.alpha);
        st->a = an;
        st->A1 = apow2(an, ian, 1.0 + mc.alpha);
        st->A3 = apow2(an, ian, 3.0 + mc.alpha);
        st->Am = apow2(an, ian, mc.alpha - 1.0);
        st->t = t + h;
        return iah;
    };
    if (kind == PK_VV_FIRST || kind == PK_VV_MID || kind == PK_VV_LAST) {
        // compact velocity-Verlet VVn (sections 5.3.2, 5.3.3): this pass closed
        // the kick of sub-step p-1 (energies E(p-1) of the synchronized momenta)
        // and opened the one of sub-step p; the next pass drifts with a_{1/2}
        double bsync = b;
        if (mc.bg) {
            bsync = bg_b(mc, t);  // prescribed background (section 4.1)
            st->hc = 0.0;
        } else {
            if (kind != PK_VV_FIRST) bsync = bh + 0.5 * pi.wc * pi.dt * Ka_u1(mc, a, EKp, EGp, EV, EKA, EGA);
            st->hc = violation(bsync, rhs(a, Et));
        }
        if (kind == PK_VV_LAST) {
            st->b = bsync;
            st->cd = 0.0;
            st->cdA = 0.0;
            return;
        }
        const double h = pi.wn * pi.dt;
        double an;
        if (mc.bg) {
            st->b = bsync;
            an = bg_a(mc, t + h);
        } else {
            const double bn = bsync + 0.5 * h * Ka_u1(mc, a, EKp, EGp, EV, EKA, EGA);
            st->bh = bn;
            an = a + h * bn;
        }
        advance(h, an);
        return;
    }
    // PK_LF: b_{+1/2} with the averaged kinetic energies (fixed point in a_{+1/2})
    if (staggered && ahm > 0)
        st->hc = violation(b, rhs(ahm, EKm0 + EKAm0 + 0.5 * (EGm0 + EGp) + 0.5 * (EVm0 + EV) + 0.5 * (EGAm0 + EGA)));
    double bp = b;
    if (mc.fmp2 > 0) {  // static background: b stays, no iteration
        for (int it = 0; it < 100; ++it) {
            const double ih = 1.0 / (a + 0.5 * pi.dt * bp), ih2 = ih * ih, ih4 = ih2 * ih2;
            const double ekp = Sp * ih4 * ih2, eka = hk * SA * ih4;
            const double bn = b + pi.dt * Ka_u1(mc, a, 0.5 * (EKm0 + ekp), EGp, EV, 0.5 * (EKAm0 + eka), EGA);
            const double d = fabs(bn - bp);
            bp = bn;
            if (d <= 1e-17 * fabs(bn) || d == 0.0) break;
        }
    }
    const double an = a + pi.dt * bp;
    const double iah = advance(pi.dt, an), ih2 = iah * iah, ih4 = ih2 * ih2;
    st->EKm = Sp * ih4 * ih2;
    st->EKAm = hk * SA * ih4;
    st->b = bp;
    st->ahm = 0.5 * (a + an);
    st->EGm = EGp; st->EVm = EV; st->EGAm = EGA;
}


}  // namespace cl
