// Batched ensembles: many independent scalar lattices (same model family,
// different coupling q, size N and seed) advanced together, one persistent
// kernel launch per integrator pass for all of them, replayed as CUDA graphs.
//
// Every member is an ordinary lattice (its own arrays, FP64 background and
// means); the ensemble kernel walks one global list of tiles (shape chosen by
// the autotuner) spanning all members.  Per tile it loads the member's
// scalars, streams the planes through the same cp.async shared-memory ring as
// the single-lattice pass, and stores the tile's sums into that member's
// per-tile partials.  A second, small kernel then sums each member's partials
// in a fixed order (one warp per member) and runs the member's FP64 background
// update (sections 4.2.3 and 4.3.2); the kernel boundary orders the partials,
// so the pass needs no memory fence or atomic per tile (a fence would wait for
// the tile's streaming stores to drain).  Members advance in lockstep through
// the same schedule of passes, with a time step common to all of them.
//
// Observations per member (workload pattern, section 4.4): the daughter-field
// energy fraction eps_chi = (E_K[chi] + E_G[chi]) / rho, the equation of state
// w = (E_K - E_G/3 - E_V)/rho, and log10 of the chi power spectrum (section 3.1)
// at 32 log-spaced momenta in [k_IR, N_min k_IR / 2], interpolated
// linearly in (log k, log Delta) between the shells of the lattice.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "cl_internal.cuh"
#include "scalar_common.cuh"

struct cl_lattice : public cl::Lattice {};

namespace cl {

struct EnsLat {
    const void* buf[2][4];  // ping-pong copies of delta phi_0, delta phi_1, delta pi_0, delta pi_1
    DevState* st;
    double* partials;  // per tile: NS sums
    ModelConst mc;
    int N, ntx, nty, ntz, ntiles, tile_base;
};

struct EnsArgs {
    const EnsLat* lat;
    const int* tile_lat;  // global tile -> member
    int ntiles;
    int src;  // copy holding the input
    int write;
    PassInfo pi;
    int BX, BY, ZC, S;
};

template <typename T, int NF, int P>
__global__ void __launch_bounds__(256, 2) ensemble_pass_kernel(const EnsArgs A) {
    constexpr int V = VecT<T>::V;
    constexpr int NS = 6 * NF + 2;
    constexpr int NA = 2 * NF;
    const int BX = A.BX, BY = A.BY, ZC = A.ZC, S = A.S;
    const int TX = BX * V, RW = TX + 2 * V, ROWS = BY + 2;
    const int ASZ = ROWS * RW, STG = NA * ASZ;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw + 128);
    __shared__ double red[8][16];
    __shared__ T* s_out[2 * NF];  // destination arrays of the tile's member
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int lin = ty * BX + tx, nthr = BX * BY;
    const int lane = lin & 31, warp = lin >> 5, nwarps = (nthr + 31) >> 5;
    const int nlanes = min(32, nthr - 32 * warp);
    const unsigned wmask = nlanes >= 32 ? 0xffffffffu : ((1u << nlanes) - 1u);
    const int dst = 1 - A.src;
    const int my_tiles = (blockIdx.x < (unsigned)A.ntiles) ? (A.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    const bool yhalo = (ty == 0) || (ty == BY - 1);
    const bool xhalo = (tx == 0) || (tx == BX - 1);
    const int yh_row = (ty == 0) ? 0 : BY + 1;
    const int xh_col = (tx == 0) ? V - 1 : V + TX;

    // producer side: member, origin and arrays of the tile being loaded
    int ld_k = 0, ld_p = 0, ld_slot = 0;
    int ld_N = 0, ld_x0 = 0, ld_y0 = 0, ld_z0 = 0;
    const T* ld_src[NA];
    auto ld_tile = [&](int k) {
        const int g = (int)blockIdx.x + k * (int)gridDim.x;
        const EnsLat& L = A.lat[A.tile_lat[g]];
        const int loc = g - L.tile_base;
        const int tyi = loc % L.nty, rr = loc / L.nty, txi = rr % L.ntx, tzi = rr / L.ntx;
        ld_N = L.N;
        ld_x0 = txi * TX;
        ld_y0 = tyi * BY;
        ld_z0 = tzi * ZC;
#pragma unroll
        for (int a = 0; a < NA; ++a) ld_src[a] = static_cast<const T*>(L.buf[A.src][a]);
    };
    if (my_tiles > 0) ld_tile(0);
    auto issue = [&]() {
        if (ld_k < my_tiles) {
            const int N = ld_N;
            int z = ld_z0 - 1 + ld_p;
            z = z < 0 ? z + N : (z >= N ? z - N : z);
            T* dstm = sm + ld_slot * STG;
            const int x = ld_x0 + tx * V, y = ld_y0 + ty;
            const size_t zoff = (size_t)z * N * N;
            const int yh = (ty == 0) ? (y == 0 ? N - 1 : y - 1) : (y == N - 1 ? 0 : y + 1);
            const int xh = (tx == 0) ? (x == 0 ? N - 1 : x - 1) : (x + V == N ? 0 : x + V);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const T* src = ld_src[a] + zoff;
                T* d = dstm + a * ASZ;
                cp_async16(d + (ty + 1) * RW + V + tx * V, src + (size_t)y * N + x);
                if (yhalo) cp_async16(d + yh_row * RW + V + tx * V, src + (size_t)yh * N + x);
                if (xhalo) cp_async_elem(d + (ty + 1) * RW + xh_col, src + (size_t)y * N + xh);
            }
            if (++ld_p == ZC + 2) {
                ld_p = 0;
                if (++ld_k < my_tiles) ld_tile(ld_k);
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
    for (int L = 0; L < S; ++L, ++issued) issue();
    int sl_m = 0, need = 2;

    for (int k = 0; k < my_tiles; ++k) {
        const int g = (int)blockIdx.x + k * (int)gridDim.x;
        const int m = A.tile_lat[g];
        const EnsLat& L = A.lat[m];
        const int N = L.N;
        const int loc = g - L.tile_base;
        const int tyi = loc % L.nty, rr = loc / L.nty, txi = rr % L.ntx, tzi = rr / L.ntx;
        const int x = txi * TX + tx * V, y = tyi * BY + ty, z0 = tzi * ZC;
        // the member's output pointers go through shared memory: read from the
        // member table inside the plane loop they would be reloaded from global
        // memory every plane (the stores may alias the table); visible after the
        // barrier of the first wait below, unused since the previous tile's end
        if (lin < NA) s_out[lin] = static_cast<T*>(const_cast<void*>(L.buf[dst][lin]));
        const DevState* st = L.st;
        const bool dead = st->error != 0;
        const T cd = T(st->cd), A1 = T(st->A1), A3 = T(st->A3);
        const T h1 = T(A.pi.h1), h = T(A.pi.h), idx2 = T(L.mc.idx2);
        const T lam = T(L.mc.lam), q = T(L.mc.q);
        T fb[2], sf[2], sp[2];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            fb[f] = f < NF ? T(st->phibar[f]) : T(0);
            sf[f] = f < NF ? T(st->sphi[f]) : T(0);
            sp[f] = f < NF ? T(st->spi[f]) : T(0);
        }
        const T P0 = fb[0] * fb[0], C0 = fb[1] * fb[1];
        const T c0[2] = {sf[0] + cd * sp[0], sf[1] + cd * sp[1]};
        const int ob = (ty + 1) * RW + V + tx * V;
        auto drift_stage = [&](T* Sx, T (&fo)[NF][V], T (&po)[NF][V]) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T* F = Sx + f * ASZ;
                const T* Pp = Sx + (NF + f) * ASZ;
                T rf[V], rp[V];
                vload_s(F + ob, rf);
                vload_s(Pp + ob, rp);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    po[f][v] = rp[v] - sp[f];
                    fo[f][v] = (rf[v] + cd * rp[v]) - c0[f];
                }
                vstore(F + ob, fo[f]);
                if (yhalo) {
                    const int oh = yh_row * RW + V + tx * V;
                    vload_s(F + oh, rf);
                    vload_s(Pp + oh, rp);
#pragma unroll
                    for (int v = 0; v < V; ++v) rf[v] = (rf[v] + cd * rp[v]) - c0[f];
                    vstore(F + oh, rf);
                }
                if (xhalo) {
                    const int oc = (ty + 1) * RW + xh_col;
                    F[oc] = (F[oc] + cd * Pp[oc]) - c0[f];
                }
            }
        };
        T ts[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) ts[i] = T(0);
        T fm[NF][V], fc[NF][V], fp[NF][V], pc[NF][V], pn[NF][V];
        // FP32: unrolled by two, the z-queue rotation is renamed away every other
        // plane (FP64 keeps the loop rolled: unrolled it would spill)
#pragma unroll(sizeof(T) == 4 ? 2 : 1)
        for (int zz = 0; zz < ZC; ++zz, ++need) {
            wait_for(need);
            if (zz > 0) { issue(); ++issued; }
            const int sl_c = sl_m + 1 == S ? 0 : sl_m + 1;
            const int sl_p = sl_c + 1 == S ? 0 : sl_c + 1;
            T* Sc = sm + sl_c * STG;
            T* Sp = sm + sl_p * STG;
            if (zz == 0) {
                T dummy[NF][V];
                drift_stage(sm + sl_m * STG, fm, dummy);
                drift_stage(Sc, fc, pc);
            }
            drift_stage(Sp, fp, pn);
            if (zz == 0) __syncthreads();
            T lap[NF][V];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T* cF = Sc + f * ASZ;
                const T fromL = __shfl_up_sync(wmask, fc[f][V - 1], 1);
                const T fromR = __shfl_down_sync(wmask, fc[f][0], 1);
                const bool useL = (tx > 0) && (lane > 0), useR = (tx < BX - 1) && (lane < nlanes - 1);
                const T left = useL ? fromL : cF[ob - 1];
                const T right = useR ? fromR : cF[ob + V];
                T u[V], d[V];
                vload_s(cF + ob - RW, u);
                vload_s(cF + ob + RW, d);
                T gs = T(0);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const T xl = (v == 0) ? left : fc[f][v - 1];
                    const T xr = (v == V - 1) ? right : fc[f][v + 1];
                    const T c = fc[f][v];
                    lap[f][v] = (((xl + xr) + (u[v] + d[v])) + (fm[f][v] + fp[f][v]) - T(6) * c) * idx2;
                    const T gx = xr - c, gy = d[v] - c, gz = fp[f][v] - c;
                    gs += gx * gx + gy * gy + gz * gz;
                }
                ts[6 * f + 4] += gs;
            }
            T pout[NF][V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T d0 = fc[0][v];
                const T d1 = NF > 1 ? fc[NF > 1 ? 1 : 0][v] : T(0);
                T F[2];
                F[0] = lam * Power<T, P>::dforce(fb[0], d0);
                F[1] = T(0);
                ts[6 * NF] += lam * Power<T, P>::dvalue(fb[0], d0);
                if (NF > 1) {
                    const T dP = d0 * (T(2) * fb[0] + d0), dC = d1 * (T(2) * fb[1] + d1);
                    F[0] += q * (C0 * d0 + dC * (fb[0] + d0));
                    F[1] = q * (P0 * d1 + dP * (fb[1] + d1));
                    ts[6 * NF + 1] += T(0.5) * q * (dP * C0 + P0 * dC + dP * dC);
                }
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T K = A1 * lap[f][v] - A3 * F[f];
                    const T pr = pc[f][v] + h1 * K;
                    pout[f][v] = pc[f][v] + h * K;
                    ts[6 * f + 0] += fc[f][v];
                    ts[6 * f + 1] += fc[f][v] * fc[f][v];
                    ts[6 * f + 2] += pr;
                    ts[6 * f + 3] += pr * pr;
                    ts[6 * f + 5] += pout[f][v];
                }
            }
            if (A.write && !dead) {
                const size_t o = ((size_t)(z0 + zz) * N + y) * N + x;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    vstore_cs(s_out[f] + o, fc[f]);
                    vstore_cs(s_out[NF + f] + o, pout[f]);
                }
            }
            sl_m = sl_m + 1 == S ? 0 : sl_m + 1;
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    fm[f][v] = fc[f][v];
                    fc[f][v] = fp[f][v];
                    pc[f][v] = pn[f][v];
                }
        }
        __syncthreads();  // the tile's last three stages are free
        issue();
        issue();
        issue();
        issued += 3;
        need += 2;
        sl_m = sl_m + 2 >= S ? sl_m + 2 - S : sl_m + 2;
        // tile sums -> the member's per-tile partials (plain stores: the finish
        // kernel that follows the pass reads them, ordered by the kernel boundary)
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const T v = partial_warp_sum(ts[i], lane, nlanes);
            if (lane == 0) red[warp][i] = double(v);
        }
        __syncthreads();
        if (lin < NS) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += red[w][lin];
            L.partials[(size_t)loc * NS + lin] = t;
        }
    }
    cp_async_wait<0>();
}


// Member finish of a pass: fixed-order compensated sums of the member's per-tile
// partials (lane l takes tiles l, l+32, ...; fixed order, then a fixed shuffle
// tree), normalised to volume averages, then the FP64 background update.
template <typename T>
__global__ void __launch_bounds__(32) ensemble_finish_kernel(const EnsLat* lat, const PassInfo pi) {
    constexpr int NS = 14;
    const EnsLat& L = lat[blockIdx.x];
    __shared__ double tot[16];
    const int lane = threadIdx.x;
    const double invV = L.mc.inv_vol;
    for (int s = 0; s < NS; ++s) {
        const double r = warp_partials_sum(L.partials, L.ntiles, NS, s, lane, 32);
        if (lane == 0) tot[s] = r * invV;
    }
    __syncwarp();
    if (lane == 0) scalar_finish(L.st, tot, L.mc, pi, sizeof(T) == 4);
}

// Observables of one lattice of the two-field model from its measured state
// and chi shell sums: the chi energy fraction (E_K[1] + E_G[1]) / rho, the
// equation of state w = (E_K - E_G/3 - E_V) / rho, and log10 of the power
// spectrum (section 3.1) interpolated linearly in (log k, log10 Delta) at 32
// log-spaced momenta between kIR and kmax (constant beyond the end shells).
void observables(const DevState& s, const double* bins, int N, double dx, double kIR, double kmax, float* o) {
    if (s.error) {
        for (int j = 0; j < CL_OBS_SIZE; ++j) o[j] = NAN;
        return;
    }
    const double EK = s.E[0] + s.E[1], EG = s.E[2] + s.E[3], EV = s.E[4] + s.E[5];
    const double rho = EK + EG + EV;
    o[0] = (float)((s.E[1] + s.E[3]) / rho);
    o[1] = (float)((EK - EG / 3.0 - EV) / rho);
    const int nb = spectrum_bins(N);
    const double norm = pow(dx / N, 3.0) / (2.0 * M_PI * M_PI);
    std::vector<double> lk, lD;
    for (int b = 1; b < nb; ++b) {
        const double c = bins[2 * (size_t)nb + b];
        if (c <= 0) continue;
        const double k = kIR * bins[(size_t)nb + b] / c;
        const double D = k * k * k * norm * bins[b] / c;
        if (D > 0) {
            lk.push_back(log(k));
            lD.push_back(log10(D));
        }
    }
    for (int j = 0; j < 32; ++j) {
        const double lkj = log(kIR) + (j + 0.5) / 32.0 * (log(kmax) - log(kIR));
        double v = NAN;
        if (!lk.empty()) {
            if (lkj <= lk.front()) v = lD.front();
            else if (lkj >= lk.back()) v = lD.back();
            else {
                const size_t u = std::upper_bound(lk.begin(), lk.end(), lkj) - lk.begin();
                const double f = (lkj - lk[u - 1]) / (lk[u] - lk[u - 1]);
                v = lD[u - 1] + f * (lD[u] - lD[u - 1]);
            }
        }
        o[2 + j] = (float)v;
    }
}

}  // namespace cl

// ------------------------------------------------------------------- host side

namespace cl {

// chi = phibar_1 + (stored - pending shift) of `count` members of one size into
// consecutive N^3 blocks (the lattice_get_field value of field 1)
template <typename T>
__global__ void ens_chi_gather_kernel(const EnsLat* lat, const int* members, int cur, size_t n3, double* out) {
    const EnsLat& L = lat[members[blockIdx.y]];
    const T* src = static_cast<const T*>(L.buf[cur][1]);
    const double mean = L.st->phibar[1];
    const T shift = T(L.st->sphi[1]);
    double* dst = out + (size_t)blockIdx.y * n3;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = mean + (double)(src[i] - shift);
}

// shell sums of |F|^2, |n~| and the mode count per member (blockIdx.y), as the
// single-lattice binning does, into bins + y * 3 * nbins
__global__ void ens_bin_kernel(const double2* F, int N, int nbins, double* bins) {
    extern __shared__ double h[];
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) h[i] = 0.0;
    __syncthreads();
    const int NH = N / 2 + 1;
    const size_t total = (size_t)N * N * NH;
    const double2* Fm = F + (size_t)blockIdx.y * total;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % NH);
        const int iy = (int)((i / NH) % N);
        const int iz = (int)(i / ((size_t)NH * N));
        const long long mx = ix, my = iy <= N / 2 ? iy : iy - N, mz = iz <= N / 2 ? iz : iz - N;
        const long long n2 = mx * mx + my * my + mz * mz;
        long long r = (long long)sqrt((double)n2);
        while ((r + 1) * (r + 1) <= n2) ++r;
        while (r * r > n2) --r;
        const int b = (int)r;
        const double w = (ix == 0 || ix == N / 2) ? 1.0 : 2.0;
        const double2 v = Fm[i];
        atomicAdd(&h[b], w * (v.x * v.x + v.y * v.y));
        atomicAdd(&h[nbins + b], w * sqrt((double)n2));
        atomicAdd(&h[2 * nbins + b], w);
    }
    __syncthreads();
    double* out = bins + (size_t)blockIdx.y * 3 * nbins;
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x)
        if (h[i] != 0.0) atomicAdd(&out[i], h[i]);
}

// every member's DevState into one array (member order)
__global__ void ens_state_gather_kernel(const EnsLat* lat, int n, DevState* out) {
    const int m = blockIdx.x;
    if (m >= n) return;
    const unsigned* src = reinterpret_cast<const unsigned*>(lat[m].st);
    unsigned* dst = reinterpret_cast<unsigned*>(out + m);
    for (size_t i = threadIdx.x; i < sizeof(DevState) / sizeof(unsigned); i += blockDim.x) dst[i] = src[i];
}

}  // namespace cl

struct cl_ensemble {
    std::vector<cl_lattice*> mem;
    std::map<int, cl::SharedFFT> fft;  // per lattice size
    cl::EnsLat* d_lat = nullptr;
    int* d_tile_lat = nullptr;
    int ntiles = 0, grid = 0, BX = 8, BY = 32, ZC = 32, S = 5;
    size_t smem = 0;
    int prec = CL_FP32, nf = 2, pexp = 2;
    int cur = 0;
    double dt = 0, kIR = 0;
    int nmin = 0;
    long long steps = 0;
    std::vector<double> weights;
    cudaStream_t stream = nullptr, cstream = nullptr;
    struct G { long long steps; int parity; int end_parity; cudaGraphExec_t exec; };
    std::vector<G> graphs;
    std::vector<cl::EnsLat> host_lat;
    int max_smem = 0;
    // batched observations: members grouped by size, chunks of at most obs_batch members
    struct ObsChunk {
        int N, first, count;   // members first .. first+count-1 of obs_members
        cufftHandle plan;      // D2Z over `count` lattices of N^3
    };
    std::vector<int> obs_members;  // member indices grouped by size
    std::vector<ObsChunk> obs_chunks;
    int* d_obs_members = nullptr;
    double* obs_in = nullptr;      // FP64 chi of one chunk
    void* obs_out = nullptr;       // its half-spectrum
    double* d_obs_bins = nullptr;  // 3 x nbins(N) per member, in obs_members order
    cl::DevState* d_obs_st = nullptr;
    std::vector<size_t> obs_bin_off;  // per position in obs_members
    size_t obs_bin_total = 0;
};

namespace {

cl_status efail(cl_status s, const std::string& m) {
    cl::set_global_error(m.c_str());
    return s;
}

const void* ens_kernel(int prec, int nf, int pexp) {
    if (nf != 2 || pexp != 2) return nullptr;
    return prec == CL_FP32 ? (const void*)cl::ensemble_pass_kernel<float, 2, 2>
                           : (const void*)cl::ensemble_pass_kernel<double, 2, 2>;
}

cudaError_t ens_launch(cl_ensemble* E, int src, const cl::PassInfo& pi, bool write, cudaStream_t s) {
    cl::EnsArgs A;
    A.lat = E->d_lat;
    A.tile_lat = E->d_tile_lat;
    A.ntiles = E->ntiles;
    A.src = src;
    A.write = write ? 1 : 0;
    A.pi = pi;
    A.BX = E->BX;
    A.BY = E->BY;
    A.ZC = E->ZC;
    A.S = E->S;
    const dim3 block(E->BX, E->BY);
    const int n = (int)E->host_lat.size();
    if (E->prec == CL_FP32) {
        cl::ensemble_pass_kernel<float, 2, 2><<<E->grid, block, E->smem, s>>>(A);
        cl::ensemble_finish_kernel<float><<<n, 32, 0, s>>>(E->d_lat, pi);
    } else {
        cl::ensemble_pass_kernel<double, 2, 2><<<E->grid, block, E->smem, s>>>(A);
        cl::ensemble_finish_kernel<double><<<n, 32, 0, s>>>(E->d_lat, pi);
    }
    return cudaGetLastError();
}

cl::PassInfo mkpass(int kind, double dt, double wc, double wn, double h1, double h) {
    cl::PassInfo p;
    p.kind = kind; p.pad = 0; p.dt = dt; p.wc = wc; p.wn = wn; p.h1 = h1; p.h = h;
    return p;
}

cudaError_t ens_enqueue(cl_ensemble* E, long long m, int* cur, cudaStream_t s) {
    const auto& w = E->weights;
    const double dt = E->dt;
    const long long S = (long long)w.size(), P = m * S;
    cudaError_t e = ens_launch(E, *cur, mkpass(cl::PK_VV_FIRST, dt, 0, w[0], 0, 0.5 * w[0] * dt), true, s);
    if (e != cudaSuccess) return e;
    *cur ^= 1;
    for (long long j = 1; j < P; ++j) {
        const double wc = w[(j - 1) % S], wn = w[j % S];
        e = ens_launch(E, *cur, mkpass(cl::PK_VV_MID, dt, wc, wn, 0.5 * wc * dt, 0.5 * (wc + wn) * dt), true, s);
        if (e != cudaSuccess) return e;
        *cur ^= 1;
    }
    const double wc = w[(P - 1) % S];
    e = ens_launch(E, *cur, mkpass(cl::PK_VV_LAST, dt, wc, 0, 0.5 * wc * dt, 0.5 * wc * dt), true, s);
    if (e != cudaSuccess) return e;
    *cur ^= 1;
    return cudaSuccess;
}

std::vector<double> ens_weights(int integ) {
    const double c = cbrt(2.0);
    if (integ == CL_INT_VV4) return {1.0 / (2.0 - c), -c / (2.0 - c), 1.0 / (2.0 - c)};
    return {1.0};
}


// A tile shape (BX, BY, ZC, S) is admissible when it divides every member,
// forms whole warps of at most 256 threads, fits the shared memory, and keeps
// each member's per-tile partial sums inside its partials array.
bool tile_ok(const cl_ensemble* E, const int32_t t[4], std::string* why) {
    const int V = E->prec == CL_FP32 ? 4 : 2, BX = t[0], BY = t[1], ZC = t[2], S = t[3];
    const int nthr = BX * BY;
    if (BX < 2 || BY < 2 || nthr % 32 != 0 || nthr > 256 || ZC < 2 || S < 4 || S > 6) {
        *why = "tile needs BX, BY >= 2, BX*BY a multiple of 32 up to 256, ZC >= 2 and 4 <= S <= 6";
        return false;
    }
    const size_t stage = 4 * (size_t)(BY + 2) * (BX * V + 2 * V) * (E->prec == CL_FP32 ? 4 : 8);
    if (128 + S * stage > (size_t)E->max_smem) {
        *why = "tile stages exceed the shared memory of a block";
        return false;
    }
    for (const auto& d : E->host_lat) {
        if (d.N % (BX * V) || d.N % BY || d.N % ZC) {
            *why = "tile does not divide N = " + std::to_string(d.N);
            return false;
        }
        const long long nt = (long long)(d.N / (BX * V)) * (d.N / BY) * (d.N / ZC);
        if (nt * 14 > (long long)cl::kMaxBlocks * cl::kMaxSums) {
            *why = "too many tiles for N = " + std::to_string(d.N) + " (take larger tiles)";
            return false;
        }
    }
    return true;
}

// installs an admissible tile shape: tile list, shared memory and persistent grid
cl_status apply_tile(cl_ensemble* E, const int32_t t[4]) {
    const int V = E->prec == CL_FP32 ? 4 : 2;
    E->BX = t[0]; E->BY = t[1]; E->ZC = t[2]; E->S = t[3];
    std::vector<int> tile_lat;
    for (size_t i = 0; i < E->host_lat.size(); ++i) {
        cl::EnsLat& d = E->host_lat[i];
        d.ntx = d.N / (E->BX * V);
        d.nty = d.N / E->BY;
        d.ntz = d.N / E->ZC;
        d.ntiles = d.ntx * d.nty * d.ntz;
        d.tile_base = (int)tile_lat.size();
        for (int k = 0; k < d.ntiles; ++k) tile_lat.push_back((int)i);
    }
    if (E->d_tile_lat) cudaFree(E->d_tile_lat);
    E->d_tile_lat = nullptr;
    E->ntiles = (int)tile_lat.size();
    if (cudaMalloc(&E->d_tile_lat, sizeof(int) * tile_lat.size()) != cudaSuccess)
        return efail(CL_ERR_OOM, "ensemble: tile list");
    cudaError_t e = cudaMemcpyAsync(E->d_lat, E->host_lat.data(), sizeof(cl::EnsLat) * E->host_lat.size(),
                                    cudaMemcpyHostToDevice, E->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E->d_tile_lat, tile_lat.data(), sizeof(int) * tile_lat.size(), cudaMemcpyHostToDevice,
                            E->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
    if (e != cudaSuccess) return efail(CL_ERR_CUDA, std::string("ensemble: tile list upload: ") + cudaGetErrorString(e));
    const size_t stage = 4 * (size_t)(E->BY + 2) * (E->BX * V + 2 * V) * (E->prec == CL_FP32 ? 4 : 8);
    E->smem = 128 + E->S * stage;
    int per_sm = 1, sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ens_kernel(E->prec, 2, 2), E->BX * E->BY, E->smem);
    if (per_sm < 1) per_sm = 1;
    E->grid = std::min(E->ntiles, sms * per_sm);
    for (auto& g : E->graphs) cudaGraphExecDestroy(g.exec);
    E->graphs.clear();
    return CL_OK;
}
}  // namespace

extern "C" {

cl_status ensemble_destroy(cl_ensemble* E) {
    if (!E) return CL_OK;
    for (auto& g : E->graphs) cudaGraphExecDestroy(g.exec);
    for (auto* L : E->mem) lattice_destroy(L);
    for (auto& kv : E->fft) {
        cufftDestroy(kv.second.c2r);
        cufftDestroy(kv.second.r2c);
        cudaFree(kv.second.work);
        cudaFree(kv.second.cwork);
    }
    if (E->d_lat) cudaFree(E->d_lat);
    if (E->d_tile_lat) cudaFree(E->d_tile_lat);
    for (auto& c : E->obs_chunks) cufftDestroy(c.plan);
    if (E->d_obs_members) cudaFree(E->d_obs_members);
    if (E->obs_in) cudaFree(E->obs_in);
    if (E->obs_out) cudaFree(E->obs_out);
    if (E->d_obs_bins) cudaFree(E->d_obs_bins);
    if (E->d_obs_st) cudaFree(E->d_obs_st);
    if (E->cstream) cudaStreamDestroy(E->cstream);
    delete E;
    return CL_OK;
}

cl_status ensemble_init(int32_t n, const cl_model* model, const double* q, const int32_t* Ns, const uint64_t* seeds,
                        const cl_grid* grid, const cl_init* init, void* cuda_stream, cl_ensemble** out) {
    if (!out) return efail(CL_ERR_ARG, "ensemble_init: out is NULL");
    *out = nullptr;
    if (n < 1 || !model || !q || !Ns || !seeds || !grid || !init)
        return efail(CL_ERR_ARG, "ensemble_init: n >= 1 and non-NULL arrays required");
    if (model->kind != CL_MODEL_SCALAR || model->n_fields != 2 || model->pexp != 2)
        return efail(CL_ERR_ARG, "ensemble_init: ensembles run the two-field model V = phi^2/2 + q phi^2 chi^2/2");
    if (grid->integrator != CL_INT_VV2 && grid->integrator != CL_INT_VV4)
        return efail(CL_ERR_ARG, "ensemble_init: ensembles run VV2 or VV4");
    for (int i = 0; i < n; ++i)
        if (Ns[i] < 32 || Ns[i] % 32 != 0 || Ns[i] > 1024 || !(q[i] >= 0))
            return efail(CL_ERR_ARG, "ensemble_init: every N must be a multiple of 32 in [32, 1024] and q >= 0");
    cl_ensemble* E = new cl_ensemble();
    E->prec = grid->precision;
    E->dt = grid->dt;
    E->kIR = grid->kIR;
    E->weights = ens_weights(grid->integrator);
    E->stream = (cudaStream_t)cuda_stream;
    E->nmin = *std::min_element(Ns, Ns + n);
    if (cudaStreamCreateWithFlags(&E->cstream, cudaStreamNonBlocking) != cudaSuccess) {
        ensemble_destroy(E);
        return efail(CL_ERR_CUDA, "ensemble_init: stream creation failed");
    }
    // shared FFT resources per lattice size
    for (int i = 0; i < n; ++i) {
        const int N = Ns[i];
        if (E->fft.count(N)) continue;
        cl::SharedFFT f{};
        const size_t n3 = (size_t)N * N * N, nh = (size_t)N * N * (N / 2 + 1);
        const bool c2r = cufftPlan3d(&f.c2r, N, N, N, CUFFT_Z2D) == CUFFT_SUCCESS;
        const bool r2c = c2r && cufftPlan3d(&f.r2c, N, N, N, CUFFT_D2Z) == CUFFT_SUCCESS;
        if (!r2c || cudaMalloc(&f.work, n3 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&f.cwork, 2 * nh * sizeof(double2)) != cudaSuccess) {
            // release what this size got before the failure (cudaFree of NULL is a no-op)
            if (c2r) cufftDestroy(f.c2r);
            if (r2c) cufftDestroy(f.r2c);
            cudaFree(f.work);
            cudaFree(f.cwork);
            ensemble_destroy(E);
            return efail(CL_ERR_OOM, "ensemble_init: FFT resources");
        }
        cufftSetStream(f.c2r, E->stream);
        cufftSetStream(f.r2c, E->stream);
        E->fft[N] = f;
    }
    // members
    for (int i = 0; i < n; ++i) {
        cl_model m = *model;
        m.q = q[i];
        cl_grid g = *grid;
        g.N = Ns[i];
        cl_init in = *init;
        in.seed = seeds[i];
        cl_lattice* L = nullptr;
        cl_status s = cl::lattice_create(&m, &g, &in, E->stream, &E->fft[Ns[i]], &L);
        if (s != CL_OK) {
            std::string msg = "ensemble_init: member " + std::to_string(i) + ": " + cl_last_error(nullptr);
            ensemble_destroy(E);
            return efail(s, msg);
        }
        E->mem.push_back(L);
    }
    // member table, then the tile list of the default shape
    for (int i = 0; i < n; ++i) {
        cl::Lattice* L = E->mem[i];
        cl::EnsLat d;
        for (int c = 0; c < 2; ++c)
            for (int a = 0; a < 4; ++a) d.buf[c][a] = L->buf.f[c][a];
        d.st = L->buf.st;
        d.partials = L->buf.partials;
        d.mc = L->mc;
        d.N = L->mc.N;
        E->host_lat.push_back(d);
    }
    if (cudaMalloc(&E->d_lat, sizeof(cl::EnsLat) * n) != cudaSuccess) {
        ensemble_destroy(E);
        return efail(CL_ERR_OOM, "ensemble_init: member table");
    }
    for (const void* fn : {(const void*)cl::ensemble_pass_kernel<float, 2, 2>, (const void*)cl::ensemble_pass_kernel<double, 2, 2>}) {
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, fn);
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const int avail = optin - (int)fa.sharedSizeBytes;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, avail);
        if (fn == ens_kernel(E->prec, 2, 2)) E->max_smem = avail;
    }
    cudaGetLastError();
    const int32_t def[4] = {E->prec == CL_FP32 ? 8 : 16, E->prec == CL_FP32 ? 32 : 16, 32, 5};
    std::string why;
    if (!tile_ok(E, def, &why)) {
        ensemble_destroy(E);
        return efail(CL_ERR_ARG, "ensemble_init: " + why);
    }
    cl_status ts = apply_tile(E, def);
    if (ts != CL_OK) {
        std::string msg = cl_last_error(nullptr);
        ensemble_destroy(E);
        return efail(ts, msg);
    }
    if (cudaStreamSynchronize(E->stream) != cudaSuccess) {
        ensemble_destroy(E);
        return efail(CL_ERR_CUDA, "ensemble_init: synchronization");
    }
    // batched observations: size classes, chunked so that one chunk's FP64 input stays under 2 GiB
    {
        std::map<int, std::vector<int>> by_size;
        for (int i = 0; i < n; ++i) by_size[Ns[i]].push_back(i);
        size_t in_max = 0, out_max = 0;
        for (auto& kv : by_size) {
            const int N = kv.first;
            const size_t n3 = (size_t)N * N * N, nh = (size_t)N * N * (N / 2 + 1);
            const int cap = (int)std::max<size_t>(1, ((size_t)1 << 31) / (n3 * sizeof(double)));
            for (size_t k = 0; k < kv.second.size(); k += cap) {
                cl_ensemble::ObsChunk c;
                c.N = N;
                c.first = (int)E->obs_members.size();
                c.count = (int)std::min<size_t>(cap, kv.second.size() - k);
                for (int m = 0; m < c.count; ++m) E->obs_members.push_back(kv.second[k + m]);
                int dims[3] = {N, N, N};
                if (cufftPlanMany(&c.plan, 3, dims, nullptr, 1, (int)n3, nullptr, 1, (int)nh, CUFFT_D2Z, c.count) !=
                    CUFFT_SUCCESS) {
                    ensemble_destroy(E);
                    return efail(CL_ERR_OOM, "ensemble_init: batched FFT plans");
                }
                cufftSetStream(c.plan, E->stream);
                E->obs_chunks.push_back(c);
                in_max = std::max(in_max, (size_t)c.count * n3);
                out_max = std::max(out_max, (size_t)c.count * nh);
            }
        }
        for (int m : E->obs_members) {
            E->obs_bin_off.push_back(E->obs_bin_total);
            E->obs_bin_total += 3 * (size_t)cl::spectrum_bins(Ns[m]);
        }
        if (cudaMalloc(&E->d_obs_members, sizeof(int) * n) != cudaSuccess ||
            cudaMalloc(&E->obs_in, sizeof(double) * in_max) != cudaSuccess ||
            cudaMalloc(&E->obs_out, sizeof(double2) * out_max) != cudaSuccess ||
            cudaMalloc(&E->d_obs_bins, sizeof(double) * E->obs_bin_total) != cudaSuccess ||
            cudaMalloc(&E->d_obs_st, sizeof(cl::DevState) * n) != cudaSuccess ||
            cudaMemcpy(E->d_obs_members, E->obs_members.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
            ensemble_destroy(E);
            return efail(CL_ERR_OOM, "ensemble_init: observation buffers");
        }
    }
    *out = E;
    return CL_OK;
}

cl_status ensemble_evolve(cl_ensemble* E, int64_t nsteps) {
    if (!E || nsteps < 0) return efail(CL_ERR_ARG, "ensemble_evolve: bad arguments");
    const long long chunk = 64;
    long long left = nsteps;
    while (left > 0) {
        const long long m = left < chunk ? left : chunk;
        cudaGraphExec_t exec = nullptr;
        int endp = E->cur;
        for (auto& g : E->graphs)
            if (g.steps == m && g.parity == E->cur) { exec = g.exec; endp = g.end_parity; }
        if (!exec) {
            int cur = E->cur;
            cudaGraph_t graph;
            if (cudaStreamBeginCapture(E->cstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return efail(CL_ERR_CUDA, "ensemble_evolve: capture");
            cudaError_t e = ens_enqueue(E, m, &cur, E->cstream);
            cudaError_t e2 = cudaStreamEndCapture(E->cstream, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) return efail(CL_ERR_CUDA, "ensemble_evolve: recording");
            if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                cudaGraphDestroy(graph);
                return efail(CL_ERR_CUDA, "ensemble_evolve: instantiate");
            }
            cudaGraphDestroy(graph);
            cl_ensemble::G g;
            g.steps = m;
            g.parity = E->cur;
            g.end_parity = cur;
            g.exec = exec;
            E->graphs.push_back(g);
            endp = cur;
        }
        if (cudaGraphLaunch(exec, E->stream) != cudaSuccess) return efail(CL_ERR_CUDA, "ensemble_evolve: launch");
        E->cur = endp;
        left -= m;
    }
    E->steps += nsteps;
    for (auto* L : E->mem) {
        L->cur = E->cur;
        L->steps_done = E->steps;
    }
    return CL_OK;
}

cl_status ensemble_member(cl_ensemble* E, int32_t i, cl_lattice** out) {
    if (!E || !out || i < 0 || i >= (int)E->mem.size()) return efail(CL_ERR_ARG, "ensemble_member: bad index");
    *out = E->mem[i];
    return CL_OK;
}

cl_status ensemble_observe(cl_ensemble* E, double kmax_arg, float* obs, double* t) {
    if (!E || !obs) return efail(CL_ERR_ARG, "ensemble_observe: NULL argument");
    const int n = (int)E->mem.size();
    // reductions of every member in one launch; then, per size class, the chi of all its
    // members gathered into one buffer, one batched D2Z and one binning launch; the
    // states and bins come back in two copies
    cudaError_t e = ens_launch(E, E->cur, mkpass(cl::PK_MEASURE, E->dt, 0, 0, 0, 0), false, E->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(E->d_obs_bins, 0, sizeof(double) * E->obs_bin_total, E->stream);
    int sm_count = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    for (const auto& c : E->obs_chunks) {
        if (e != cudaSuccess) break;
        const int N = c.N;
        const size_t n3 = (size_t)N * N * N;
        const int nb = cl::spectrum_bins(N);
        const int gx = std::max(1, std::min(64, (int)((n3 + 255) / 256)));
        const dim3 g(gx, c.count);
        if (E->prec == CL_FP32)
            cl::ens_chi_gather_kernel<float><<<g, 256, 0, E->stream>>>(E->d_lat, E->d_obs_members + c.first, E->cur, n3,
                                                                       E->obs_in);
        else
            cl::ens_chi_gather_kernel<double><<<g, 256, 0, E->stream>>>(E->d_lat, E->d_obs_members + c.first, E->cur, n3,
                                                                        E->obs_in);
        e = cudaGetLastError();
        if (e == cudaSuccess && cufftExecD2Z(c.plan, E->obs_in, (cufftDoubleComplex*)E->obs_out) != CUFFT_SUCCESS)
            e = cudaErrorUnknown;
        if (e == cudaSuccess) {
            const size_t nh = (size_t)N * N * (N / 2 + 1);
            const int bx = std::max(1, std::min(2 * sm_count, (int)((nh + 511) / 512)));
            cl::ens_bin_kernel<<<dim3(bx, c.count), 512, 3 * (size_t)nb * sizeof(double), E->stream>>>(
                (const double2*)E->obs_out, N, nb, E->d_obs_bins + E->obs_bin_off[c.first]);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        cl::ens_state_gather_kernel<<<n, 128, 0, E->stream>>>(E->d_lat, n, E->d_obs_st);
        e = cudaGetLastError();
    }
    std::vector<cl::DevState> st(n);
    std::vector<double> bins(E->obs_bin_total);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st.data(), E->d_obs_st, sizeof(cl::DevState) * n, cudaMemcpyDeviceToHost, E->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bins.data(), E->d_obs_bins, sizeof(double) * bins.size(), cudaMemcpyDeviceToHost, E->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
    if (e != cudaSuccess) return efail(CL_ERR_CUDA, std::string("ensemble_observe: ") + cudaGetErrorString(e));
    const double kmax = kmax_arg > 0 ? kmax_arg : 0.5 * E->nmin * E->kIR;
    for (size_t k = 0; k < E->obs_members.size(); ++k) {
        const int i = E->obs_members[k];
        cl::observables(st[i], bins.data() + E->obs_bin_off[k], E->mem[i]->mc.N, E->mem[i]->mc.dx, E->kIR, kmax,
                        obs + (size_t)i * CL_OBS_SIZE);
    }
    if (t) *t = st.empty() ? 0.0 : st[0].t;
    return CL_OK;
}

cl_status ensemble_get_tile(const cl_ensemble* E, int32_t tile[4]) {
    if (!E || !tile) return efail(CL_ERR_ARG, "ensemble_get_tile: NULL argument");
    tile[0] = E->BX; tile[1] = E->BY; tile[2] = E->ZC; tile[3] = E->S;
    return CL_OK;
}

cl_status ensemble_set_tile(cl_ensemble* E, const int32_t tile[4]) {
    if (!E || !tile) return efail(CL_ERR_ARG, "ensemble_set_tile: NULL argument");
    std::string why;
    if (!tile_ok(E, tile, &why)) return efail(CL_ERR_ARG, "ensemble_set_tile: " + why);
    return apply_tile(E, tile);
}

cl_status ensemble_autotune(cl_ensemble* E, int32_t max_report, int32_t* tiles, double* ms, int32_t* n_tried) {
    if (!E || max_report < 0) return efail(CL_ERR_ARG, "ensemble_autotune: bad arguments");
    static const int32_t c32[][4] = {{8, 32, 32, 5}, {8, 32, 16, 5}, {8, 32, 32, 4}, {8, 16, 32, 4}, {8, 16, 32, 5},
                                     {8, 16, 32, 6}, {8, 16, 16, 5}, {8, 8, 32, 5},  {8, 8, 32, 6},  {16, 16, 32, 5},
                                     {16, 8, 32, 5}, {4, 32, 32, 5}};
    static const int32_t c64[][4] = {{16, 16, 32, 5}, {16, 16, 16, 5}, {16, 16, 32, 4}, {16, 8, 32, 5}, {16, 8, 32, 6},
                                     {8, 32, 32, 5},  {8, 16, 32, 5},  {16, 16, 8, 5},  {8, 8, 32, 5},  {16, 4, 32, 5},
                                     {32, 8, 32, 5},  {4, 32, 32, 5}};
    const int nc = 12;
    const int32_t(*cand)[4] = E->prec == CL_FP32 ? c32 : c64;
    const int n = (int)E->mem.size();
    const int32_t keep[4] = {E->BX, E->BY, E->ZC, E->S};
    // snapshot of every member's scalar state: the timing passes write only the
    // spare copy of the fields, so restoring the states undoes them
    cl::DevState* snap = nullptr;
    if (cudaMalloc(&snap, sizeof(cl::DevState) * n) != cudaSuccess) return efail(CL_ERR_OOM, "ensemble_autotune");
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(snap + i, E->mem[i]->buf.st, sizeof(cl::DevState), cudaMemcpyDeviceToDevice, E->stream);
    auto restore = [&]() {
        for (int i = 0; i < n && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(E->mem[i]->buf.st, snap + i, sizeof(cl::DevState), cudaMemcpyDeviceToDevice, E->stream);
    };
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    const double w0 = E->weights[0], dt = E->dt;
    const cl::PassInfo pass = mkpass(cl::PK_VV_MID, dt, w0, w0, 0.5 * w0 * dt, w0 * dt);
    int best = -1, tried = 0;
    float best_ms = 0;
    cl_status st = CL_OK;
    for (int c = 0; c < nc && e == cudaSuccess && st == CL_OK; ++c) {
        std::string why;
        if (!tile_ok(E, cand[c], &why)) continue;
        st = apply_tile(E, cand[c]);
        if (st != CL_OK) break;
        const int reps = 3;
        e = ens_launch(E, E->cur, pass, true, E->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev0, E->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = ens_launch(E, E->cur, pass, true, E->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, E->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
        float t = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev0, ev1);
        restore();
        t /= reps;
        if (tried < max_report) {
            if (tiles)
                for (int j = 0; j < 4; ++j) tiles[4 * tried + j] = cand[c][j];
            if (ms) ms[tried] = t;
        }
        ++tried;
        if (best < 0 || t < best_ms) {
            best = c;
            best_ms = t;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaFree(snap);
    if (n_tried) *n_tried = tried;
    if (st != CL_OK) return st;
    if (e != cudaSuccess) return efail(CL_ERR_CUDA, std::string("ensemble_autotune: ") + cudaGetErrorString(e));
    return apply_tile(E, best >= 0 ? cand[best] : keep);
}

}  // extern "C"
