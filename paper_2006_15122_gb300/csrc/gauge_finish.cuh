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

static __device__ double Ka_u1(const ModelConst& mc, double a, double EKp, double EGp, double EV, double EKA, double EGA) {
    return mc.fmp2 / 3.0 * apow(a, 2.0 * mc.alpha + 1.0) *
           ((mc.alpha - 2.0) * EKp + mc.alpha * EGp + (mc.alpha + 1.0) * EV + (mc.alpha - 1.0) * (EKA + EGA));
}

// SU(2) x U(1) + chi (ns = 15) adds {<sum piA_sync^2>, <sum_{i<j} (1 - cos theta_ij)>,
// <pchi_sync^2>, <sum_i (D_i^+ chi)^2>/dx^2}; the background update then sees the
// scalar sectors (Phi, chi) and the gauge sectors (SU(2), U(1)) in aggregate,
// which is exact because every energy of one class scales with the same power
// of a (chi's kinetic and gradient energies carry the 1/2 of a real field).
static __device__ void u1_finish(DevState* st, const double* tot, const ModelConst& mc, const PassInfo& pi,
                                 int ns = U1NS) {
    const double a = st->a, a2 = a * a, a4 = a2 * a2, a6 = a4 * a2;
    const double dx4 = mc.dx * mc.dx * mc.dx * mc.dx;
    double Sp = tot[6], SA = tot[9], SG = tot[7], SM = tot[10] / (mc.e * mc.e);
    if (ns > U1NS) {
        Sp += 0.5 * tot[13];
        SG += 0.5 * tot[14];
        if (mc.e2 > 0) {
            SA += tot[11];
            SM += tot[12] / (mc.e2 * mc.e2);
        }
    }
    const double EKp = Sp / a6, EGp = SG / a2, EV = tot[8];
    const double EKA = mc.kappa * SA / (2.0 * a4), EGA = mc.kappa * SM / (a4 * dx4);
    st->E[0] = EKp; st->E[1] = EGp; st->E[2] = EV; st->E[3] = EKA; st->E[4] = EGA;
    for (int s = 0; s < ns; ++s) st->sums[s] = tot[s];
    const double Et = EKp + EGp + EV + EKA + EGA;
    if (!isfinite(Et)) { st->error = CL_ERR_NONFINITE; return; }
    auto rhs = [&](double aa, double E) { return mc.fmp2 / 3.0 * apow(aa, 2.0 * (mc.alpha + 1.0)) * E; };
    const int kind = pi.kind;
    if (kind == PK_MEASURE) {
        if (mc.bg) {
            st->hc = 0.0;
        } else if (st->staggered) {
            const double r = rhs(st->ahm, st->EKm + st->EKAm + 0.5 * (st->EGm + EGp) + 0.5 * (st->EVm + EV) +
                                              0.5 * (st->EGAm + EGA));
            st->hc = r > 0 ? fabs(st->b * st->b - r) / r : 0.0;
        } else {
            const double r = rhs(a, Et);
            st->hc = r > 0 ? fabs(st->b * st->b - r) / r : 0.0;
        }
        return;
    }
    if (kind == PK_INIT_B) {
        if (mc.bg) st->b = bg_b(mc, st->t);
        else st->b = mc.fmp2 > 0 ? sqrt(fmax(rhs(a, Et), 0.0)) : 0.0;
        st->hc = 0.0;
        return;
    }
    if (kind == PK_LF_EKM) {
        st->EKm = Sp / apow(st->ahm, 6.0);
        st->EKAm = mc.kappa * SA / (2.0 * apow(st->ahm, 4.0));
        return;
    }
    if (kind == PK_LF_PREPARE) {
        const double bm = st->b - 0.5 * pi.dt * Ka_u1(mc, a, EKp, EGp, EV, EKA, EGA);
        st->b = bm;
        st->ahm = a - 0.5 * pi.dt * bm;
        st->EGm = EGp; st->EVm = EV; st->EGAm = EGA;
        st->staggered = 1;
        st->cd = 0.0;
        st->cdA = 0.0;
        return;
    }
    if (kind == PK_VV_FIRST || kind == PK_VV_MID || kind == PK_VV_LAST) {
        // compact velocity-Verlet VVn (sections 5.3.2, 5.3.3): this pass closed
        // the kick of sub-step p-1 (energies E(p-1) of the synchronized momenta)
        // and opened the one of sub-step p; the next pass drifts with a_{1/2}
        double bsync = st->b;
        if (mc.bg) {
            bsync = bg_b(mc, st->t);  // prescribed background (section 4.1)
            st->hc = 0.0;
        } else {
            if (kind != PK_VV_FIRST) bsync = st->bh + 0.5 * pi.wc * pi.dt * Ka_u1(mc, a, EKp, EGp, EV, EKA, EGA);
            const double r = rhs(a, Et);
            st->hc = r > 0 ? fabs(bsync * bsync - r) / r : 0.0;
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
            an = bg_a(mc, st->t + h);
        } else {
            const double bn = bsync + 0.5 * h * Ka_u1(mc, a, EKp, EGp, EV, EKA, EGA);
            st->bh = bn;
            an = a + h * bn;
        }
        const double ah = 0.5 * (a + an);
        st->cd = h * apow(ah, -(3.0 - mc.alpha));
        st->cdA = mc.e * mc.dx * h * apow(ah, -(1.0 - mc.alpha));
        st->a = an;
        st->A1 = apow(an, 1.0 + mc.alpha);
        st->A3 = apow(an, 3.0 + mc.alpha);
        st->Am = apow(an, mc.alpha - 1.0);
        st->t += h;
        return;
    }
    // PK_LF: b_{+1/2} with the averaged kinetic energies (fixed point in a_{+1/2})
    if (st->staggered && st->ahm > 0) {
        const double r = rhs(st->ahm, st->EKm + st->EKAm + 0.5 * (st->EGm + EGp) + 0.5 * (st->EVm + EV) +
                                          0.5 * (st->EGAm + EGA));
        st->hc = r > 0 ? fabs(st->b * st->b - r) / r : 0.0;
    }
    double bp = st->b, ekp = 0, eka = 0;
    for (int it = 0; it < 100; ++it) {
        const double ah = a + 0.5 * pi.dt * bp;
        ekp = Sp / apow(ah, 6.0);
        eka = mc.kappa * SA / (2.0 * apow(ah, 4.0));
        const double bn = st->b + pi.dt * Ka_u1(mc, a, 0.5 * (st->EKm + ekp), EGp, EV, 0.5 * (st->EKAm + eka), EGA);
        const double d = fabs(bn - bp);
        bp = bn;
        if (d <= 1e-17 * fabs(bn) || d == 0.0) break;
    }
    const double an = a + pi.dt * bp, ah = 0.5 * (a + an);
    st->EKm = Sp / apow(ah, 6.0);
    st->EKAm = mc.kappa * SA / (2.0 * apow(ah, 4.0));
    st->b = bp;
    st->ahm = ah;
    st->EGm = EGp; st->EVm = EV; st->EGAm = EGA;
    st->cd = pi.dt * apow(ah, -(3.0 - mc.alpha));
    st->cdA = mc.e * mc.dx * pi.dt * apow(ah, -(1.0 - mc.alpha));
    st->a = an;
    st->A1 = apow(an, 1.0 + mc.alpha);
    st->A3 = apow(an, 3.0 + mc.alpha);
    st->Am = apow(an, mc.alpha - 1.0);
    st->t += pi.dt;
}


}  // namespace cl
