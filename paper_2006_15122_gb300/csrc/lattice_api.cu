// C ABI of the lattice library (include/cl_lattice.h): handle life cycle,
// integrator schedules recorded as CUDA graphs, measurements, checkpoints.
//
// Integrator schedules (paper sections 4.2.1, 4.2.3, 4.3.2, 5.3.1) as
// sequences of fused passes, each "drift (prepared by the previous pass),
// then kick, then reductions":
//   VVn, n steps of s sub-steps with weights w_p:
//     pass 0       kick w_1 dt/2                         (E at the start)
//     pass j       drift w_p dt, kick (w_p + w_{p+1}) dt/2 (merged half kicks)
//     pass n*s     drift w_s dt, kick w_s dt/2            (synchronizes)
//   leapfrog, n steps: n passes "drift dt, kick dt" plus one closing drift;
//   a backward half kick starts it from synchronized data.
// The drift coefficient w dt a_{1/2}^{-(3-alpha)} and the next a come from
// the Friedmann update that the last block of each pass performs, so a whole
// evolve call runs without the host.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "cl_internal.cuh"

struct cl_lattice : public cl::Lattice {};

namespace {

thread_local std::string g_err = "no error";

cl_status fail(cl::Lattice* L, cl_status s, const std::string& msg) {
    if (L) L->err = msg;
    else g_err = msg;
    return s;
}

cl_status cuda_fail(cl::Lattice* L, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(L, e == cudaErrorMemoryAllocation ? CL_ERR_OOM : CL_ERR_CUDA, m);
}

// Weights of the Yoshida compositions (section 4.3.2; appendix table).  VV4 in
// closed form: w1 = w3 = 1/(2 - 2^(1/3)), w2 = -2^(1/3)/(2 - 2^(1/3)).
std::vector<double> yoshida(int integ) {
    const double c = cbrt(2.0);
    std::vector<double> h;
    switch (integ) {
        case CL_INT_LF:
        case CL_INT_VV2: return {1.0};
        case CL_INT_VV4: return {1.0 / (2.0 - c), -c / (2.0 - c), 1.0 / (2.0 - c)};
        case CL_INT_VV6:
            h = {0.78451361047755726382, 0.23557321335935813368, -1.1776799841788710069, 1.3151863206839112189};
            break;
        case CL_INT_VV8:
            h = {0.74167036435061295345, -0.40910082580003159400, 0.19075471029623837995, -0.57386247111608226666,
                 0.29906418130365592384, 0.33462491824529818378,  0.31529309239676659663, -0.79688793935291635402};
            break;
        case CL_INT_VV10:
            h = {-0.48159895600253002870, 0.0036303931544595926879, 0.50180317558723140279, 0.28298402624506254868,
                 0.80702967895372223806,  -0.026090580538592205447, -0.87286590146318071547, -0.52373568062510581643,
                 0.44521844299952789252,  0.18612289547097907887,   0.23137327866438360633, -0.52191036590418628905,
                 0.74866113714499296793,  0.066736511890604057532,  -0.80360324375670830316, 0.91249037635867994571};
            break;
        default: return {};
    }
    std::vector<double> w(h);
    for (int i = (int)h.size() - 2; i >= 0; --i) w.push_back(h[i]);
    return w;
}

// Largest x = omega dt for which the composed velocity-Verlet map of a
// harmonic mode stays stable (|trace| < 2) on all of (0, x].
double stability_limit(const std::vector<double>& w) {
    const double dx = 1e-4;
    for (double x = dx; x < 8.0; x += dx) {
        double m00 = 1, m01 = 0, m10 = 0, m11 = 1;
        for (double wi : w) {
            const double hx = wi * x, c = 1 - 0.5 * hx * hx;
            const double a00 = c, a01 = hx, a10 = -hx * (1 - 0.25 * hx * hx), a11 = c;
            const double n00 = a00 * m00 + a01 * m10, n01 = a00 * m01 + a01 * m11;
            const double n10 = a10 * m00 + a11 * m10, n11 = a10 * m01 + a11 * m11;
            m00 = n00; m01 = n01; m10 = n10; m11 = n11;
        }
        if (fabs(m00 + m11) >= 2.0) return x - dx;
    }
    return 8.0;
}

cudaError_t launch_pass(cl::Lattice* L, int src, int dst, const cl::PassInfo& pi, bool write, cudaStream_t s) {
    if (L->mc.kind == CL_MODEL_SCALAR) return cl::scalar_launch_pass(L, src, dst, pi, write, s);
    if (L->mc.kind == CL_MODEL_SU2) return cl::su2_launch_pass(L, src, dst, pi, write, s);
    return cl::u1_launch_pass(L, src, dst, pi, write, s);
}

cudaError_t launch_drift(cl::Lattice* L, int cur, cudaStream_t s) {
    cudaError_t e = L->mc.kind == CL_MODEL_SCALAR ? cl::scalar_launch_drift(L, cur, s)
                    : L->mc.kind == CL_MODEL_SU2  ? cl::su2_launch_drift(L, cur, s)
                                                  : cl::u1_launch_drift(L, cur, s);
    if (e != cudaSuccess) return e;
    return cl::launch_finish_drift(L, s);
}

cl::PassInfo make_pass(int kind, double dt, double wc, double wn, double h1, double h) {
    cl::PassInfo p;
    p.kind = kind;
    p.pad = 0;
    p.dt = dt;
    p.wc = wc;
    p.wn = wn;
    p.h1 = h1;
    p.h = h;
    return p;
}

// Parts of one evolve call that is recorded as several graphs: the passes of
// a long call are one sequence, cut into graphs of at most 64 steps without
// synchronizing the state at the cuts (no extra pass per graph).
enum GraphPart : int {
    GP_WHOLE = 0,  // the whole call: opening kick ... closing kick (or closing drift)
    GP_HEAD = 1,   // opens the call, ends inside it
    GP_BODY = 2,   // starts and ends inside the call
    GP_TAIL = 3    // starts inside the call and closes it
};

// Enqueue m steps starting from copy `cur`; returns the copy holding the result.
// `part` selects whether this piece opens (GP_WHOLE, GP_HEAD) and closes
// (GP_WHOLE, GP_TAIL) the evolve call; RK4 and Gauss-Legendre steps are
// self-contained and take every piece as whole.
cudaError_t enqueue_steps(cl::Lattice* L, long long m, int* cur, cudaStream_t s, int part) {
    const double dt = L->grid.dt;
    if (L->integ == CL_INT_RK4) return cl::rk4_enqueue(L, m, *cur, s);  // the state stays in copy `cur`
    if (L->integ >= CL_INT_GL2) return cl::gl_enqueue(L, m, *cur, s);
    const bool opens = part == GP_WHOLE || part == GP_HEAD, closes = part == GP_WHOLE || part == GP_TAIL;
    if (L->integ == CL_INT_LF) {
        for (long long j = 0; j < m; ++j) {
            cudaError_t e = launch_pass(L, *cur, 1 - *cur, make_pass(cl::PK_LF, dt, 0, 0, dt, dt), true, s);
            if (e != cudaSuccess) return e;
            *cur ^= 1;
        }
        return closes ? launch_drift(L, *cur, s) : cudaSuccess;
    }
    // VVn: global pass j of the call (j = 0 the opening kick, j = 1.. merged
    // kicks with wc = w[(j-1) mod S], wn = w[j mod S]); a piece that does not
    // open the call starts at a merged kick whose wc is the last weight.
    const std::vector<double>& w = L->weights;
    const long long S = (long long)w.size(), P = m * S;
    cudaError_t e = cudaSuccess;
    long long j0 = 0;
    if (opens) {
        e = launch_pass(L, *cur, 1 - *cur, make_pass(cl::PK_VV_FIRST, dt, 0, w[0], 0, 0.5 * w[0] * dt), true, s);
        if (e != cudaSuccess) return e;
        *cur ^= 1;
        j0 = 1;
    }
    for (long long j = j0; j < P; ++j) {
        const double wc = w[(j + S - 1) % S], wn = w[j % S];
        e = launch_pass(L, *cur, 1 - *cur, make_pass(cl::PK_VV_MID, dt, wc, wn, 0.5 * wc * dt, 0.5 * (wc + wn) * dt), true, s);
        if (e != cudaSuccess) return e;
        *cur ^= 1;
    }
    if (!closes) return cudaSuccess;
    const double wc = w[S - 1];
    e = launch_pass(L, *cur, 1 - *cur, make_pass(cl::PK_VV_LAST, dt, wc, 0, 0.5 * wc * dt, 0.5 * wc * dt), true, s);
    if (e != cudaSuccess) return e;
    *cur ^= 1;
    return cudaSuccess;
}

cl_status ensure_staggered(cl::Lattice* L) {
    if (L->integ != CL_INT_LF || L->staggered) return CL_OK;
    const double dt = L->grid.dt;
    cudaError_t e = launch_pass(L, L->cur, 1 - L->cur, make_pass(cl::PK_LF_PREPARE, dt, 0, 0, 0, -0.5 * dt), true, L->stream);
    if (e != cudaSuccess) return cuda_fail(L, e, "leapfrog start");
    L->cur ^= 1;
    e = launch_pass(L, L->cur, 1 - L->cur, make_pass(cl::PK_LF_EKM, dt, 0, 0, 0, 0), false, L->stream);
    if (e != cudaSuccess) return cuda_fail(L, e, "leapfrog start");
    L->staggered = true;
    return CL_OK;
}

cudaGraphExec_t get_graph(cl::Lattice* L, long long m, int parity, int part, cudaError_t* err) {
    for (auto& g : L->graphs)
        if (g.steps == m && g.parity == parity && g.part == part) return g.exec;
    int cur = parity;
    cudaGraph_t graph;
    *err = cudaStreamBeginCapture(L->cstream, cudaStreamCaptureModeThreadLocal);
    if (*err != cudaSuccess) return nullptr;
    cudaError_t e = enqueue_steps(L, m, &cur, L->cstream, part);
    cudaError_t e2 = cudaStreamEndCapture(L->cstream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        *err = e != cudaSuccess ? e : e2;
        return nullptr;
    }
    cudaGraphExec_t exec;
    *err = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (*err != cudaSuccess) return nullptr;
    cl::Lattice::G g;
    g.steps = m;
    g.parity = parity;
    g.part = part;
    g.exec = exec;
    g.end_parity = cur;
    L->graphs.push_back(g);
    return exec;
}

int graph_end_parity(cl::Lattice* L, long long m, int parity, int part) {
    for (auto& g : L->graphs)
        if (g.steps == m && g.parity == parity && g.part == part) return g.end_parity;
    return parity;
}

uint32_t crc32_update(uint32_t crc, const unsigned char* p, size_t n) {
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

// Bound on the curvature of the gauge models' potential at the homogeneous
// start, mod2 = |phi|^2 = S/2 with S the squared canonical norm: along a
// canonical component chi it is dV/dmod2 + chi^2 d^2V/dmod2^2, at most
// |dV/dmod2| + 2 mod2 |d^2V/dmod2^2|.
double gauge_m2_bound(const cl::ModelConst& mc, double mod2) {
    double dv;
    cl::gauge_pot<double>(mc.gpot, mc.pexp, mc.lam, mc.vev2, mod2, &dv);
    return fabs(dv) + 2.0 * mod2 * fabs(cl::gauge_pot_d2(mc.gpot, mc.pexp, mc.lam, mod2));
}

struct CkptHeader {
    char magic[8];
    int32_t version, prec, narr, staggered;
    cl_model model;
    cl_grid grid;
    cl_init init;
    int64_t steps;
    uint64_t nbytes;
    uint32_t crc;
    uint32_t pad;
};

}  // namespace

namespace cl {
// Records the reason of a failure that has no handle (reported by cl_last_error(NULL)).
void set_global_error(const char* msg) { g_err = msg; }
}  // namespace cl

extern "C" {

const char* cl_status_str(cl_status s) {
    switch (s) {
        case CL_OK: return "ok";
        case CL_ERR_ARG: return "invalid argument";
        case CL_ERR_CUDA: return "CUDA error";
        case CL_ERR_OOM: return "out of device memory";
        case CL_ERR_UNSTABLE_DT: return "time step beyond the integrator's stability bound";
        case CL_ERR_NONFINITE: return "non-finite value in a reduction";
        case CL_ERR_TIMEOUT: return "timeout";
        case CL_ERR_STATE: return "call does not fit the handle's state";
        case CL_ERR_IO: return "checkpoint I/O or verification error";
    }
    return "unknown status";
}

const char* cl_last_error(const cl_lattice* h) { return h ? h->err.c_str() : g_err.c_str(); }

int32_t lattice_spectrum_bins(const cl_lattice* h) { return h ? cl::spectrum_bins(h->mc.N) : 0; }

cl_status lattice_destroy(cl_lattice* h) {
    if (!h) return CL_OK;
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < cl::kMaxArrays; ++i)
            if (h->buf.f[c][i]) cudaFree(h->buf.f[c][i]);
    for (int i = 0; i < 4; ++i) {
        if (h->rk_T1[i]) cudaFree(h->rk_T1[i]);
        if (h->rk_A[i]) cudaFree(h->rk_A[i]);
        for (int b = 0; b < 2; ++b)
            for (int l = 0; l < 5; ++l)
                if (h->gl_D[b][l][i]) cudaFree(h->gl_D[b][l][i]);
    }
    if (h->buf.st) cudaFree(h->buf.st);
    if (h->buf.partials) cudaFree(h->buf.partials);
    if (h->buf.counter) cudaFree(h->buf.counter);
    if (h->bins) cudaFree(h->bins);
    if (!h->shared_fft) {
        if (h->work) cudaFree(h->work);
        if (h->cwork) cudaFree(h->cwork);
        if (h->plans) {
            cufftDestroy(h->plan_c2r);
            cufftDestroy(h->plan_r2c);
        }
    }
    if (h->cstream) cudaStreamDestroy(h->cstream);
    delete h;
    return CL_OK;
}

cl_status lattice_init(const cl_model* model, const cl_grid* grid, const cl_init* init, void* cuda_stream,
                       cl_lattice** out) {
    return cl::lattice_create(model, grid, init, (cudaStream_t)cuda_stream, nullptr, out);
}

}  // extern "C"

cl_status cl::lattice_create(const cl_model* model, const cl_grid* grid, const cl_init* init, cudaStream_t cuda_stream,
                             const cl::SharedFFT* shared, cl_lattice** out) {
    if (!out) return fail(nullptr, CL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!model || !grid || !init) return fail(nullptr, CL_ERR_ARG, "model, grid and init must be non-NULL");
    const int N = grid->N;
    if (N < 8 || N > 2048 || N % 8 != 0) return fail(nullptr, CL_ERR_ARG, "N must be a multiple of 8 in [8, 2048]");
    if (!(grid->kIR > 0) || !(grid->dt > 0) || !isfinite(grid->dt)) return fail(nullptr, CL_ERR_ARG, "kIR and dt must be positive");
    if (grid->precision != CL_FP64 && grid->precision != CL_FP32) return fail(nullptr, CL_ERR_ARG, "unknown precision");
    if (model->kind == CL_MODEL_SCALAR) {
        if (model->n_fields < 1 || model->n_fields > 2) return fail(nullptr, CL_ERR_ARG, "n_fields must be 1 or 2");
        if (model->pexp != 2 && model->pexp != 4 && model->pexp != 6) return fail(nullptr, CL_ERR_ARG, "pexp must be 2, 4 or 6");
        if (grid->integrator < CL_INT_LF || grid->integrator > CL_INT_GL5) return fail(nullptr, CL_ERR_ARG, "unknown integrator");
        if (grid->integrator >= CL_INT_RK4 && (grid->precision != CL_FP64 || model->background != CL_BG_FRIEDMANN))
            return fail(nullptr, CL_ERR_ARG, "RK4 and Gauss-Legendre run in FP64 with the self-consistent background");
    } else if (model->kind == CL_MODEL_U1 || model->kind == CL_MODEL_SU2) {
        if (grid->integrator < CL_INT_LF || grid->integrator > CL_INT_VV10) return fail(nullptr, CL_ERR_ARG, "unknown integrator");
        if (!(model->gauge_e > 0)) return fail(nullptr, CL_ERR_ARG, "gauge_e must be positive");
        if (model->potential != CL_POT_HIGGS && model->potential != CL_POT_MONOMIAL)
            return fail(nullptr, CL_ERR_ARG, "unknown gauge potential");
        if (model->noncompact != 0 && (model->noncompact != 1 || model->kind != CL_MODEL_U1))
            return fail(nullptr, CL_ERR_ARG, "noncompact is 0, or 1 for the U(1) model");
        // the U(1) pass indexes sites in 32 bits (its 20 arrays of N^3 would not fit in memory beyond that)
        if (model->kind == CL_MODEL_U1 && (long long)N * N * N >= (1LL << 32))
            return fail(nullptr, CL_ERR_ARG, "U(1): N^3 must be below 2^32");
        if (model->potential == CL_POT_MONOMIAL && model->pexp != 2 && model->pexp != 4 && model->pexp != 6)
            return fail(nullptr, CL_ERR_ARG, "pexp must be 2, 4 or 6");
        if (model->kind == CL_MODEL_SU2) {
            if (model->n_fields != 1 && model->n_fields != 2)
                return fail(nullptr, CL_ERR_ARG, "SU(2): n_fields is 1, or 2 with the singlet chi");
            if (!(model->gauge_e_u1 >= 0) || !isfinite(model->gauge_e_u1))
                return fail(nullptr, CL_ERR_ARG, "gauge_e_u1 must be >= 0");
            // ... and the U(1) charge Im[Phi^dag pi]
            if (model->gauge_e_u1 > 0) {
                const double* f = init->phi0;
                const double* p = init->dphi0;
                const double q0 = f[0] * p[1] - f[1] * p[0] + f[2] * p[3] - f[3] * p[2];
                if (fabs(q0) > 1e-12 * (1.0 + fabs(f[0]) + fabs(f[1]) + fabs(f[2]) + fabs(f[3])))
                    return fail(nullptr, CL_ERR_ARG, "the homogeneous U(1) charge Im[Phi^dag Phi'] must vanish");
            }
            // a uniform charge Im[Phi^dag sigma^a pi] cannot satisfy the Gauss law on a periodic lattice
            const double* f = init->phi0;
            const double* p = init->dphi0;
            const double q1 = f[0] * p[3] - f[1] * p[2] + f[2] * p[1] - f[3] * p[0];
            const double q2 = -f[0] * p[2] - f[1] * p[3] + f[2] * p[0] + f[3] * p[1];
            const double q3 = f[0] * p[1] - f[1] * p[0] - f[2] * p[3] + f[3] * p[2];
            if (fabs(q1) + fabs(q2) + fabs(q3) > 1e-12 * (1.0 + fabs(f[0]) + fabs(f[1]) + fabs(f[2]) + fabs(f[3])))
                return fail(nullptr, CL_ERR_ARG, "the homogeneous SU(2) charge Im[Phi^dag sigma^a Phi'] must vanish");
        }
    } else {
        return fail(nullptr, CL_ERR_ARG, "unknown model kind");
    }
    if (!(model->omega_over_fstar > 0)) return fail(nullptr, CL_ERR_ARG, "omega_over_fstar must be positive");
    if (model->background != CL_BG_FRIEDMANN && model->background != CL_BG_FLUID)
        return fail(nullptr, CL_ERR_ARG, "unknown background");
    if (model->background == CL_BG_FLUID) {
        const double den = 3.0 * (1.0 + model->fluid_w) - 2.0 * model->alpha;
        if (!(den > 0) || !isfinite(model->fluid_w) || !(model->hubble0 >= 0) || !isfinite(model->hubble0))
            return fail(nullptr, CL_ERR_ARG, "fluid background needs 3(1 + w) - 2 alpha > 0 and hubble0 >= 0");
        if (grid->integrator == CL_INT_LF || model->kind != CL_MODEL_SCALAR)
            return fail(nullptr, CL_ERR_ARG, "the fluid background runs the scalar model under velocity-Verlet");
    }
    if (init->a0 < 0 || !isfinite(init->a0)) return fail(nullptr, CL_ERR_ARG, "a0 must be positive (0 selects 1)");

    cl_lattice* L = new cl_lattice();
    memset(L->buf.f, 0, sizeof(L->buf.f));
    memset(L->rk_T1, 0, sizeof(L->rk_T1));
    memset(L->rk_A, 0, sizeof(L->rk_A));
    memset(L->gl_D, 0, sizeof(L->gl_D));
    L->buf.st = nullptr; L->buf.partials = nullptr; L->buf.counter = nullptr;
    L->work = nullptr; L->cwork = nullptr; L->bins = nullptr; L->plans = false; L->cstream = nullptr;
    L->shared_fft = shared != nullptr;
    L->grid = *grid;
    L->init = *init;
    if (!(L->init.a0 > 0)) L->init.a0 = 1.0;
    if (!(L->init.fluct_scale > 0)) L->init.fluct_scale = init->spectrum ? 1.0 : 0.0;
    L->integ = grid->integrator;
    L->prec = grid->precision;
    L->tsize = L->prec == CL_FP32 ? 4 : 8;
    L->stream = (cudaStream_t)cuda_stream;
    L->cur = 0;
    L->steps_done = 0;
    L->staggered = false;
    L->weights = yoshida(L->integ);
    cl::ModelConst& mc = L->mc;
    mc.kind = model->kind;
    mc.nf = model->kind == CL_MODEL_SCALAR ? model->n_fields : 2;
    mc.pexp = model->pexp;
    mc.N = N;
    mc.alpha = model->alpha;
    mc.fmp2 = model->fstar_over_mp * model->fstar_over_mp;
    mc.lam = model->lam;
    mc.q = model->q;
    mc.vev2 = model->vev2;
    mc.e = model->gauge_e;
    mc.kappa = model->omega_over_fstar * model->omega_over_fstar;
    mc.dx = 2.0 * M_PI / (grid->kIR * N);
    mc.idx2 = 1.0 / (mc.dx * mc.dx);
    mc.gpot = mc.kind == CL_MODEL_SCALAR ? 0 : model->potential;
    mc.e2 = mc.kind == CL_MODEL_SU2 ? model->gauge_e_u1 : 0.0;
    mc.chi = mc.kind == CL_MODEL_SU2 && model->n_fields == 2 ? 1 : 0;
    mc.ext = mc.e2 > 0 || mc.chi ? 1 : 0;
    mc.nc = mc.kind == CL_MODEL_U1 && model->noncompact ? 1 : 0;
    mc.bg = model->background == CL_BG_FLUID ? 1 : 0;
    mc.bg_p = mc.bg ? 2.0 / (3.0 * (1.0 + model->fluid_w) - 2.0 * model->alpha) : 1.0;
    mc.bg_H0 = mc.bg ? model->hubble0 : 0.0;
    mc.bg_a0 = L->init.a0;
    mc.fmp2_3 = mc.fmp2 / 3.0;
    mc.inv_vol = 1.0 / ((double)N * N * N);
    mc.inv_e_sq = mc.e > 0 ? 1.0 / (mc.e * mc.e) : 0.0;
    mc.inv_e2_sq = mc.e2 > 0 ? 1.0 / (mc.e2 * mc.e2) : 0.0;
    mc.inv_dx4 = mc.idx2 * mc.idx2;

    // linear stability of the highest lattice mode
    {
        const double a = L->init.a0;
        double m2 = 0.0;
        if (mc.kind == CL_MODEL_SCALAR) {
            const double f0 = init->phi0[0], f1 = mc.nf > 1 ? init->phi0[1] : 0.0;
            double ap = 1.0;
            for (int i = 0; i < mc.pexp - 2; ++i) ap *= fabs(f0);
            m2 = std::max(fabs((mc.pexp - 1) * mc.lam * ap + (mc.nf > 1 ? mc.q * f1 * f1 : 0.0)),
                          mc.nf > 1 ? fabs(mc.q * f0 * f0) : 0.0);
        } else if (mc.kind == CL_MODEL_SU2) {
            double s2 = 0.0;
            for (int c = 0; c < 4; ++c) s2 += init->phi0[c] * init->phi0[c];
            // gauge masses g^2 |Phi|^2/(2 kappa) and (U(1)) 2 eA^2 |Phi|^2/kappa bound the mixed mass matrix;
            // the singlet's curvature is 2 q |Phi|^2
            m2 = gauge_m2_bound(mc, s2) + mc.e * mc.e * s2 / (2.0 * mc.kappa) + 2.0 * mc.e2 * mc.e2 * s2 / mc.kappa;
            if (mc.chi) m2 = std::max(m2, fabs(2.0 * mc.q * s2));
        } else {
            const double s2 = 0.5 * (init->phi0[0] * init->phi0[0] + init->phi0[1] * init->phi0[1]);
            m2 = gauge_m2_bound(mc, s2) + 2.0 * mc.e * mc.e * s2 / mc.kappa;
        }
        const double w2 = pow(a, 2.0 * mc.alpha - 2.0) * 12.0 * mc.idx2 + pow(a, 2.0 * mc.alpha) * m2;
        // RK4: the stability interval of the oscillator on the imaginary axis is |w dt| < 2 sqrt(2)
        // Gauss-Legendre is A-stable; the bound 2 keeps its fixed-point stage iteration contracting
        const double lim = L->integ == CL_INT_RK4 ? 2.8 : (L->integ >= CL_INT_GL2 ? 2.0 : stability_limit(L->weights));
        if (!grid->force_dt && sqrt(w2) * grid->dt >= lim) {
            char msg[256];
            snprintf(msg, sizeof msg, "omega_max dt = %.4g exceeds the stability bound %.4g of this integrator",
                     sqrt(w2) * grid->dt, lim);
            delete L;
            return fail(nullptr, CL_ERR_UNSTABLE_DT, msg);
        }
    }

    cudaError_t e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&L->sm_count, cudaDevAttrMultiProcessorCount, dev);
    L->buf.narr = 0;
    if (cl::array_count(mc) > cl::kMaxArrays) {
        cl_status s = fail(nullptr, CL_ERR_ARG, "internal: more stored arrays than the handle holds");
        lattice_destroy(L);
        return s;
    }
    L->buf.narr = cl::array_count(mc);
    const size_t n = (size_t)N * N * N;
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < L->buf.narr; ++i) {
            e = cudaMalloc(&L->buf.f[c][i], n * L->tsize);
            if (e != cudaSuccess) { cl_status s = cuda_fail(nullptr, e, "allocating fields"); lattice_destroy(L); return s; }
        }
    if (L->integ >= CL_INT_GL2)
        for (int b = 0; b < 2; ++b)
            for (int l = 0; l < L->integ - CL_INT_GL2 + 2; ++l)
                for (int i = 0; i < L->buf.narr; ++i)
                    if ((e = cudaMalloc(&L->gl_D[b][l][i], n * sizeof(double))) != cudaSuccess) {
                        cl_status s = cuda_fail(nullptr, e, "allocating Gauss-Legendre stages");
                        lattice_destroy(L);
                        return s;
                    }
    if (L->integ == CL_INT_RK4)
        for (int i = 0; i < L->buf.narr; ++i)
            if ((e = cudaMalloc(&L->rk_T1[i], n * sizeof(double))) != cudaSuccess ||
                (e = cudaMalloc(&L->rk_A[i], n * sizeof(double))) != cudaSuccess) {
                cl_status s = cuda_fail(nullptr, e, "allocating RK4 stages");
                lattice_destroy(L);
                return s;
            }
    const size_t nh = (size_t)N * N * (N / 2 + 1);
    if ((e = cudaMalloc(&L->buf.st, sizeof(cl::DevState))) != cudaSuccess ||
        (e = cudaMalloc(&L->buf.partials, sizeof(double) * cl::kMaxBlocks * cl::kMaxSums)) != cudaSuccess ||
        (e = cudaMalloc(&L->buf.counter, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&L->cstream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&L->bins, 3 * sizeof(double) * (size_t)lattice_spectrum_bins(L))) != cudaSuccess ||
        (!shared && ((e = cudaMalloc(&L->work, n * sizeof(double))) != cudaSuccess ||
                     (e = cudaMalloc(&L->cwork, 2 * nh * sizeof(double2))) != cudaSuccess))) {
        cl_status s = cuda_fail(nullptr, e, "allocating scratch");
        lattice_destroy(L);
        return s;
    }
    cudaMemsetAsync(L->buf.counter, 0, sizeof(unsigned int), L->stream);
    cudaMemsetAsync(L->buf.st, 0, sizeof(cl::DevState), L->stream);
    if (shared) {
        L->plan_c2r = shared->c2r;
        L->plan_r2c = shared->r2c;
        L->work = shared->work;
        L->cwork = shared->cwork;
        L->plans = true;
    } else {
        if (cufftPlan3d(&L->plan_c2r, N, N, N, CUFFT_Z2D) != CUFFT_SUCCESS ||
            cufftPlan3d(&L->plan_r2c, N, N, N, CUFFT_D2Z) != CUFFT_SUCCESS) {
            lattice_destroy(L);
            return fail(nullptr, CL_ERR_CUDA, "cuFFT plan creation failed");
        }
        L->plans = true;
        cufftSetStream(L->plan_c2r, L->stream);
        cufftSetStream(L->plan_r2c, L->stream);
    }
    if (mc.kind == CL_MODEL_SCALAR) cl::scalar_geometry(L);
    else if (mc.kind == CL_MODEL_SU2) cl::su2_geometry(L);
    else cl::u1_geometry(L);

    cl_status s = cl::ic_generate(L);
    if (s != CL_OK) {
        std::string m = "initial conditions: " + std::string(cudaGetErrorString(cudaGetLastError()));
        lattice_destroy(L);
        return fail(nullptr, s, m);
    }
    e = launch_pass(L, L->cur, 1 - L->cur, make_pass(cl::PK_INIT_B, grid->dt, 0, 0, 0, 0), false, L->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) {
        cl_status s2 = cuda_fail(nullptr, e, "initial Hubble rate");
        lattice_destroy(L);
        return s2;
    }
    *out = L;
    return CL_OK;
}

extern "C" {

cl_status lattice_evolve(cl_lattice* h, int64_t nsteps) {
    if (!h) return fail(nullptr, CL_ERR_ARG, "NULL handle");
    if (nsteps < 0) return fail(h, CL_ERR_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return CL_OK;
    cl_status s = ensure_staggered(h);
    if (s != CL_OK) return s;
    // Graphs of at most 64 steps; the pieces of one call continue each other's
    // pass sequence, so a call of n velocity-Verlet steps runs n*s + 1 passes.
    const long long chunk = 64;
    long long left = nsteps;
    bool first = true;
    while (left > 0) {
        const long long m = left < chunk ? left : chunk;
        const bool last = m == left;
        const int part = first ? (last ? GP_WHOLE : GP_HEAD) : (last ? GP_TAIL : GP_BODY);
        cudaError_t e = cudaSuccess;
        cudaGraphExec_t g = get_graph(h, m, h->cur, part, &e);
        if (!g) return cuda_fail(h, e, "recording the evolve graph");
        e = cudaGraphLaunch(g, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "launching the evolve graph");
        h->cur = graph_end_parity(h, m, h->cur, part);
        left -= m;
        first = false;
    }
    h->steps_done += nsteps;
    return CL_OK;
}

static cl_status read_state(cl_lattice* h, cl::DevState* st) {
    cudaError_t e = cudaMemcpyAsync(st, h->buf.st, sizeof(*st), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reading the device state");
    if (st->error == CL_ERR_TIMEOUT)
        return fail(h, CL_ERR_TIMEOUT,
                    "the Gauss-Legendre stage equations did not converge within 60 sweeps; the lattice stopped at "
                    "the last completed step");
    if (st->error == cl::kErrCopyTimeout)
        return fail(h, CL_ERR_TIMEOUT, "a field pass gave up waiting for its tensor copies; the lattice stopped");
    if (st->error) return fail(h, CL_ERR_NONFINITE, "a reduction produced a non-finite value; the lattice stopped");
    return CL_OK;
}

cl_status lattice_measure_means(cl_lattice* h, cl_means* out) {
    if (!h || !out) return fail(h, CL_ERR_ARG, "NULL argument");
    cudaError_t e = launch_pass(h, h->cur, 1 - h->cur, make_pass(cl::PK_MEASURE, h->grid.dt, 0, 0, 0, 0), false, h->stream);
    if (e == cudaSuccess && h->mc.kind == CL_MODEL_U1) e = cl::u1_launch_gauss(h, h->cur, h->stream);
    if (e == cudaSuccess && h->mc.kind == CL_MODEL_SU2) e = cl::su2_launch_gauss(h, h->cur, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "measure pass");
    cl::DevState st;
    cl_status s = read_state(h, &st);
    if (s != CL_OK) return s;
    memset(out, 0, sizeof(*out));
    out->t = st.t;
    out->a = st.a;
    out->b = st.b;
    out->step = h->steps_done;
    if (h->mc.kind == CL_MODEL_SCALAR) {
        const int nf = h->mc.nf;
        double EKt = 0, EGt = 0;
        for (int f = 0; f < nf; ++f) {
            const double m1 = st.sums[6 * f + 0], m2 = st.sums[6 * f + 1];
            out->mean[f] = st.phibar[f] + m1;
            out->mean2[f] = st.phibar[f] * st.phibar[f] + 2.0 * st.phibar[f] * m1 + m2;
            out->var[f] = m2 - m1 * m1;
            out->mean_pi[f] = st.pibar[f] + st.sums[6 * f + 2];
            out->EK[f] = st.E[f];
            out->EG[f] = st.E[2 + f];
            EKt += st.E[f];
            EGt += st.E[2 + f];
        }
        if (h->staggered) {
            EKt = st.EKm;
            out->EK[0] = st.EKm;
            out->EK[1] = 0.0;
            out->reserved[0] = 1.0;  // EK[0] holds the total kinetic energy at t - dt/2
        }
        out->EV[0] = st.E[4];
        out->EV[1] = st.E[5];
        const double EVt = st.E[4] + st.E[5];
        out->rho = EKt + EGt + EVt;
        out->w = out->rho != 0 ? (EKt - EGt / 3.0 - EVt) / out->rho : 0.0;
    } else {
        for (int c = 0; c < 2; ++c) {
            out->mean[c] = st.sums[c];
            out->mean2[c] = st.sums[2 + c];
            out->var[c] = st.sums[2 + c] - st.sums[c] * st.sums[c];
            out->mean_pi[c] = st.sums[4 + c];
        }
        const double EKp = h->staggered ? st.EKm : st.E[0], EKA = h->staggered ? st.EKAm : st.E[3];
        out->EK[0] = EKp; out->EK[1] = EKA;
        out->EG[0] = st.E[1]; out->EG[1] = st.E[4];
        out->EV[0] = st.E[2];
        if (h->mc.ext) {
            // per sector from the sums of the last pass (st.E holds the scalar and gauge aggregates);
            // under the leapfrog the kinetic entries EK[0], EK[1] keep the aggregates at t - dt/2
            const cl::ModelConst& mc = h->mc;
            const double a = st.a, a2 = a * a, a4 = a2 * a2, a6 = a4 * a2, dx4 = mc.dx * mc.dx * mc.dx * mc.dx;
            const double* S = st.sums;
            if (!h->staggered) {
                out->EK[0] = S[6] / a6;
                out->EK[1] = mc.kappa * S[9] / (2.0 * a4);
                out->EK[2] = mc.e2 > 0 ? mc.kappa * S[11] / (2.0 * a4) : 0.0;
                out->EK[3] = mc.chi ? 0.5 * S[13] / a6 : 0.0;
            }
            out->EG[0] = S[7] / a2;
            out->EG[1] = mc.kappa * S[10] / (a4 * mc.e * mc.e * dx4);
            out->EG[2] = mc.e2 > 0 ? mc.kappa * S[12] / (a4 * mc.e2 * mc.e2 * dx4) : 0.0;
            out->EG[3] = mc.chi ? 0.5 * S[14] / a2 : 0.0;
            out->EV[0] = st.E[2];
        }
        out->rho = EKp + EKA + st.E[1] + st.E[2] + st.E[4];
        // scalar p = K - G/3 - V; gauge radiation p = (E_K^A + E_G^A)/3
        const double p = EKp - st.E[1] / 3.0 - st.E[2] + (EKA + st.E[4]) / 3.0;
        out->w = out->rho != 0 ? p / out->rho : 0.0;
        const double den = st.gauss[1] + st.gauss[2];
        out->gauss_violation = den > 0 ? sqrt(st.gauss[0]) / sqrt(den) : sqrt(st.gauss[0]);
    }
    out->hubble_violation = st.hc;
    return CL_OK;
}

cl_status lattice_observe(cl_lattice* h, double kmax, float* obs, double* t) {
    if (!h || !obs) return fail(h, CL_ERR_ARG, "NULL argument");
    if (h->mc.kind != CL_MODEL_SCALAR || h->mc.nf != 2 || h->staggered)
        return fail(h, CL_ERR_ARG, "observables need the two-field scalar model under a velocity-Verlet integrator");
    if (!(kmax > 0)) kmax = 0.5 * h->mc.N * h->grid.kIR;
    cudaError_t e = launch_pass(h, h->cur, 1 - h->cur, make_pass(cl::PK_MEASURE, h->grid.dt, 0, 0, 0, 0), false, h->stream);
    if (e == cudaSuccess) e = cl::launch_spectrum(h, 1, 0, h->stream);
    cl::DevState st;
    std::vector<double> hb(3 * (size_t)cl::spectrum_bins(h->mc.N));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, h->buf.st, sizeof(st), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb.data(), h->bins, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "observables");
    cl::observables(st, hb.data(), h->mc.N, h->mc.dx, h->grid.kIR, kmax, obs);
    if (t) *t = st.t;
    return CL_OK;
}

cl_status lattice_measure_gauge_spectrum(cl_lattice* h, int32_t sector, int32_t what, double* k, double* Delta,
                                         int64_t* counts) {
    if (!h || !k || !Delta || !counts) return fail(h, CL_ERR_ARG, "NULL argument");
    if (what != 0 && what != 1) return fail(h, CL_ERR_ARG, "what must be 0 (electric) or 1 (magnetic)");
    const bool u1 = h->mc.kind == CL_MODEL_U1 || (h->mc.kind == CL_MODEL_SU2 && h->mc.e2 > 0);
    if (sector == 0 ? !u1 : (sector != 1 || h->mc.kind != CL_MODEL_SU2))
        return fail(h, CL_ERR_ARG, "this model has no such gauge sector");
    int ncomp = 0;
    cudaError_t e = cl::launch_gauge_spectrum(h, sector, what, &ncomp, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "gauge spectrum");
    cl::DevState st;
    cl_status s = read_state(h, &st);
    if (s != CL_OK) return s;
    const int nb = lattice_spectrum_bins(h);
    std::vector<double> hb(3 * (size_t)nb);
    e = cudaMemcpyAsync(hb.data(), h->bins, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "gauge spectrum readback");
    const double N = h->mc.N, dx = h->mc.dx;
    // E_i = piA_i / a^{1-alpha} (E_i^a = piB_i^a / a^{1-alpha})
    const double scale = what == 0 ? pow(st.a, 2.0 * h->mc.alpha - 2.0) : 1.0;
    const double norm = pow(dx / N, 3.0) / (2.0 * M_PI * M_PI) * scale;
    for (int b = 0; b < nb; ++b) {
        const double c = hb[2 * (size_t)nb + b] / (double)ncomp;
        counts[b] = (int64_t)llround(c);
        const double mean_n = c > 0 ? hb[(size_t)nb + b] / (double)ncomp / c : 0.0;
        k[b] = h->grid.kIR * mean_n;
        Delta[b] = c > 0 ? k[b] * k[b] * k[b] * norm * hb[b] / c : 0.0;
    }
    return CL_OK;
}

cl_status lattice_measure_spectrum(cl_lattice* h, int32_t field, int32_t what, double* k, double* Delta,
                                   int64_t* counts) {
    if (!h || !k || !Delta || !counts) return fail(h, CL_ERR_ARG, "NULL argument");
    if (what != 0 && what != 1) return fail(h, CL_ERR_ARG, "what must be 0 (field) or 1 (momentum)");
    std::vector<int> slots;
    if (h->mc.kind == CL_MODEL_SCALAR) {
        if (field < 0 || field >= h->mc.nf) return fail(h, CL_ERR_ARG, "field index out of range");
        slots.push_back(what == 0 ? field : h->mc.nf + field);
    } else if (h->mc.kind == CL_MODEL_SU2) {  // the doublet: spectra summed over its four components
        if (field == 1 && h->mc.chi) {
            slots.push_back(what == 0 ? 35 : 36);  // the singlet
        } else {
            if (field != 0) return fail(h, CL_ERR_ARG, "the SU(2) model has one doublet (index 0) and the singlet (1)");
            for (int c = 0; c < 4; ++c) slots.push_back(what == 0 ? c : 4 + c);
        }
    } else {
        if (field != 0) return fail(h, CL_ERR_ARG, "the U(1) model has one complex field (index 0)");
        slots.push_back(what == 0 ? 0 : 2);
        slots.push_back(what == 0 ? 1 : 3);
    }
    for (size_t i = 0; i < slots.size(); ++i) {
        cudaError_t e = cl::launch_spectrum(h, slots[i], i > 0, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "spectrum");
    }
    const int nb = lattice_spectrum_bins(h);
    std::vector<double> hb(3 * (size_t)nb);
    cudaError_t e = cudaMemcpyAsync(hb.data(), h->bins, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "spectrum readback");
    const double N = h->mc.N, dx = h->mc.dx;
    const double norm = pow(dx / N, 3.0) / (2.0 * M_PI * M_PI);
    for (int b = 0; b < nb; ++b) {
        const double c = hb[2 * (size_t)nb + b] / (double)slots.size();
        counts[b] = (int64_t)llround(c);
        const double mean_n = c > 0 ? hb[(size_t)nb + b] / (double)slots.size() / c : 0.0;
        k[b] = h->grid.kIR * mean_n;
        Delta[b] = c > 0 ? k[b] * k[b] * k[b] * norm * hb[b] / c : 0.0;
    }
    return CL_OK;
}

cl_status lattice_get_field(cl_lattice* h, int32_t which, double* dst, int32_t on_device) {
    if (!h || !dst) return fail(h, CL_ERR_ARG, "NULL argument");
    const int slot = cl::array_slot(h->mc, which);
    if (slot < 0) return fail(h, CL_ERR_ARG, "array index out of range for this model");
    const size_t n = (size_t)h->mc.N * h->mc.N * h->mc.N;
    cudaError_t e = cl::launch_get_field(h, slot, on_device ? dst : h->work, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(dst, h->work, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_field");
    return CL_OK;
}

cl_status lattice_set_field(cl_lattice* h, int32_t which, const double* src, int32_t on_device) {
    if (!h || !src) return fail(h, CL_ERR_ARG, "NULL argument");
    const int slot = cl::array_slot(h->mc, which);
    if (slot < 0) return fail(h, CL_ERR_ARG, "array index out of range for this model");
    const size_t n = (size_t)h->mc.N * h->mc.N * h->mc.N;
    const double* s = src;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        e = cudaMemcpyAsync(h->work, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        s = h->work;
    }
    if (e == cudaSuccess) e = cl::launch_set_field(h, slot, s, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);  // host buffer may go away
    if (e != cudaSuccess) return cuda_fail(h, e, "set_field");
    return CL_OK;
}

cl_status lattice_get_stored(cl_lattice* h, int32_t which, void* dst, double* mean, int32_t on_device) {
    if (!h || !dst || !mean) return fail(h, CL_ERR_ARG, "NULL argument");
    const int slot = cl::array_slot(h->mc, which);
    if (slot < 0) return fail(h, CL_ERR_ARG, "array index out of range for this model");
    const size_t n = (size_t)h->mc.N * h->mc.N * h->mc.N;
    const size_t bytes = n * (h->prec == CL_FP32 ? sizeof(float) : sizeof(double));
    // device scratch: the N^3-double work array holds either precision; its mean after it
    double* mean_dev = h->bins;
    cudaError_t e = cl::launch_get_stored(h, slot, on_device ? dst : (void*)h->work, mean_dev, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(dst, h->work, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mean, mean_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_stored");
    return CL_OK;
}

cl_status lattice_set_stored(cl_lattice* h, int32_t which, const void* src, double mean, int32_t on_device) {
    if (!h || !src) return fail(h, CL_ERR_ARG, "NULL argument");
    const int slot = cl::array_slot(h->mc, which);
    if (slot < 0) return fail(h, CL_ERR_ARG, "array index out of range for this model");
    if (!isfinite(mean)) return fail(h, CL_ERR_ARG, "mean must be finite");
    if (!cl::has_mean(h->mc, slot) && mean != 0.0)
        return fail(h, CL_ERR_ARG, "this array has no homogeneous part: mean must be 0");
    const size_t n = (size_t)h->mc.N * h->mc.N * h->mc.N;
    const size_t bytes = n * (h->prec == CL_FP32 ? sizeof(float) : sizeof(double));
    cudaError_t e = cudaMemcpyAsync(h->buf.f[h->cur][slot], src, bytes,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cl::launch_set_stored_mean(h, slot, mean, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);  // host buffer may go away
    if (e != cudaSuccess) return cuda_fail(h, e, "set_stored");
    return CL_OK;
}

}  // extern "C"

namespace {
__global__ void set_background_kernel(cl::DevState* st, double a, double b, double t, double alpha) {
    st->a = a;
    st->b = b;
    st->t = t;
    st->bh = 0.0;
    st->cd = 0.0;
    st->cdA = 0.0;
    st->A1 = pow(a, 1.0 + alpha);
    st->A3 = pow(a, 3.0 + alpha);
    st->Am = pow(a, alpha - 1.0);
    st->staggered = 0;
    st->error = 0;
    for (int f = 0; f < cl::kMaxComp; ++f) st->sphi[f] = 0.0;
}
}  // namespace

extern "C" cl_status lattice_set_background(cl_lattice* h, double a, double b, double t) {
    if (!h) return fail(nullptr, CL_ERR_ARG, "NULL handle");
    if (h->mc.bg) {  // prescribed background: a and b follow t
        if (!isfinite(t)) return fail(h, CL_ERR_ARG, "t must be finite");
        a = cl::bg_a(h->mc, t);
        b = cl::bg_b(h->mc, t);
    }
    if (!(a > 0) || !isfinite(a)) return fail(h, CL_ERR_ARG, "a must be positive");
    // a pending leapfrog drift is never left between calls, so shifts of phi are already applied
    set_background_kernel<<<1, 1, 0, h->stream>>>(h->buf.st, a, isnan(b) ? 0.0 : b, t, h->mc.alpha);
    cudaError_t e = cudaGetLastError();
    // a pass that stopped on an error may have left its block counter part-way
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf.counter, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess && isnan(b))
        e = launch_pass(h, h->cur, 1 - h->cur, make_pass(cl::PK_INIT_B, h->grid.dt, 0, 0, 0, 0), false, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_background");
    h->staggered = false;
    return CL_OK;
}

extern "C" cl_status lattice_save(cl_lattice* h, const char* path) {
    if (!h || !path) return fail(h, CL_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->mc.N * h->mc.N * h->mc.N;
    std::vector<unsigned char> st(sizeof(cl::DevState));
    cudaError_t e = cudaMemcpyAsync(st.data(), h->buf.st, st.size(), cudaMemcpyDeviceToHost, h->stream);
    std::vector<unsigned char> arr(n * h->tsize);
    CkptHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, "CLLAT001", 8);
    hd.version = 1;
    hd.prec = h->prec;
    hd.narr = h->buf.narr;
    hd.staggered = h->staggered ? 1 : 0;
    hd.grid = h->grid;
    hd.init = h->init;
    hd.model.kind = h->mc.kind;
    hd.model.n_fields = h->mc.nf;
    hd.model.pexp = h->mc.pexp;
    hd.model.alpha = h->mc.alpha;
    hd.model.lam = h->mc.lam;
    hd.model.q = h->mc.q;
    hd.model.vev2 = h->mc.vev2;
    hd.model.gauge_e = h->mc.e;
    hd.model.fstar_over_mp = sqrt(h->mc.fmp2);
    hd.model.omega_over_fstar = sqrt(h->mc.kappa);
    hd.model.potential = h->mc.gpot;
    hd.model.gauge_e_u1 = h->mc.e2;
    hd.model.noncompact = h->mc.nc;
    if (h->mc.kind == CL_MODEL_SU2) hd.model.n_fields = h->mc.chi ? 2 : 1;
    hd.steps = h->steps_done;
    hd.nbytes = st.size() + (uint64_t)h->buf.narr * arr.size();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint readback");
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(h, CL_ERR_IO, std::string("cannot open ") + path);
    uint32_t crc = crc32_update(0, st.data(), st.size());
    bool ok = fwrite(&hd, sizeof hd, 1, fp) == 1 && fwrite(st.data(), 1, st.size(), fp) == st.size();
    for (int i = 0; ok && i < h->buf.narr; ++i) {
        e = cudaMemcpy(arr.data(), h->buf.f[h->cur][i], arr.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { fclose(fp); return cuda_fail(h, e, "checkpoint readback"); }
        crc = crc32_update(crc, arr.data(), arr.size());
        ok = fwrite(arr.data(), 1, arr.size(), fp) == arr.size();
    }
    hd.crc = crc;
    ok = ok && fseek(fp, 0, SEEK_SET) == 0 && fwrite(&hd, sizeof hd, 1, fp) == 1;
    ok = (fclose(fp) == 0) && ok;
    if (!ok) return fail(h, CL_ERR_IO, std::string("short write to ") + path);
    return CL_OK;
}

extern "C" cl_status lattice_restore(cl_lattice* h, const char* path) {
    if (!h || !path) return fail(h, CL_ERR_ARG, "NULL argument");
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(h, CL_ERR_IO, std::string("cannot open ") + path);
    CkptHeader hd;
    if (fread(&hd, sizeof hd, 1, fp) != 1 || memcmp(hd.magic, "CLLAT001", 8) != 0 || hd.version != 1) {
        fclose(fp);
        return fail(h, CL_ERR_IO, "not a lattice checkpoint");
    }
    if (hd.prec != h->prec || hd.narr != h->buf.narr || hd.grid.N != h->mc.N || hd.model.kind != h->mc.kind ||
        hd.model.n_fields != (h->mc.kind == CL_MODEL_SU2 ? (h->mc.chi ? 2 : 1) : h->mc.nf) ||
        hd.grid.integrator != h->integ) {
        fclose(fp);
        return fail(h, CL_ERR_IO, "checkpoint of another geometry, model, integrator or precision");
    }
    const size_t n = (size_t)h->mc.N * h->mc.N * h->mc.N;
    std::vector<unsigned char> st(sizeof(cl::DevState));
    std::vector<std::vector<unsigned char>> arrs(h->buf.narr, std::vector<unsigned char>(n * h->tsize));
    bool ok = fread(st.data(), 1, st.size(), fp) == st.size();
    uint32_t crc = crc32_update(0, st.data(), st.size());
    for (int i = 0; ok && i < h->buf.narr; ++i) {
        ok = fread(arrs[i].data(), 1, arrs[i].size(), fp) == arrs[i].size();
        crc = crc32_update(crc, arrs[i].data(), arrs[i].size());
    }
    fclose(fp);
    if (!ok) return fail(h, CL_ERR_IO, "truncated checkpoint");
    if (crc != hd.crc) return fail(h, CL_ERR_IO, "checkpoint CRC mismatch");
    cudaError_t e = cudaMemcpy(h->buf.st, st.data(), st.size(), cudaMemcpyHostToDevice);
    for (int i = 0; e == cudaSuccess && i < h->buf.narr; ++i)
        e = cudaMemcpy(h->buf.f[h->cur][i], arrs[i].data(), arrs[i].size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint upload");
    h->steps_done = hd.steps;
    h->staggered = hd.staggered != 0;
    return CL_OK;
}
