// Fused scalar-sector pass for sm_103a: drift -> 7-point Laplacian -> kick ->
// volume reductions, one HBM read and one HBM write of every array per pass.
//
// Method (paper sections 4.2.1, 4.2.3, 4.3.2, Hamiltonian form):
//   phi_i' = a^{-(3-alpha)} pi_i,
//   pi_i'  = K_i = a^{1+alpha} L[phi_i] - a^{3+alpha} dV/dphi_i,
//   L[f](n) = sum_k (f(n+k) + f(n-k) - 2 f(n)) / dx^2,
//   b' = K_a = (1/3)(f*/m_p)^2 a^{1+2alpha} [(alpha-2) E_K + alpha E_G + (alpha+1) E_V],
//   E_K = sum_i <pi_i^2>/(2a^6), E_G = sum_{i,k} <(D_k^+ phi_i)^2>/(2a^2), E_V = <V>,
// with V = (lam/p)|phi|^p + (q/2) phi^2 chi^2 (section 8.1).
//
// One pass applies the drift that the previous pass prepared (its coefficient
// needs the previous pass's volume averages through a(eta)), then the kick
// K evaluated on the drifted fields, and reduces in the same sweep the sums
// that give E_K, E_G, E_V and the means.  Adjacent half kicks of consecutive
// velocity-Verlet sub-steps are merged into one kick; the kinetic energy of
// the synchronized momenta (first half kick only) is formed in registers.
// The last block to finish sums the per-block partials in a fixed order and
// advances a, b and the homogeneous means in FP64 (last-block-done pattern),
// so consecutive passes need no host round trip.
//
// Mean/fluctuation split: each field is phibar (FP64, in DevState) + delta
// (array of T).  The kick of the mean is -a^{3+alpha} V'(phibar) in FP64; the
// array gets a^{1+alpha} L[delta] - a^{3+alpha} [V'(phibar+delta) - V'(phibar)]
// written as a polynomial in delta, so no large number is ever subtracted
// in FP32.  The volume mean that the fluctuations pick up is moved into
// phibar/pibar after every pass (a pending shift subtracted on the next
// read), which keeps phi = phibar + delta exact.
//
// Tiling: a block of BX x BY threads owns a tile of BX*V x BY sites in x-y
// (V = 4 floats or 2 doubles per thread, 16-byte accesses) and marches ZC
// planes in z; z-neighbours live in registers, x-y neighbours of the drifted
// plane in shared memory (double-buffered, one barrier per plane), halo
// cells are loaded by the tile-edge threads.  Loads of plane z+2 and of the
// halo of plane z+1 are issued before the compute of plane z.  The grid is
// persistent (grid-stride over tiles, y-tiles fastest so that y-halos are
// L2 hits of concurrently running tiles).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "cl_internal.cuh"
#include "scalar_common.cuh"

namespace cl {

struct ScalarArgs {
    const void* in[4];  // slots 0..nf-1: delta phi, nf..2nf-1: delta pi (source copy)
    void* out[4];       // same slots, destination copy
    DevState* st;
    double* partials;
    unsigned int* counter;
    ModelConst mc;
    Geometry geo;
    PassInfo pi;
    int write;
};

// --------------------------------------------------------------- the pass

struct TileXYZ {
    int x0, y0, z0;
};

__device__ __forceinline__ TileXYZ decode_tile(const Geometry& g, int tile) {
    const int tyi = tile % g.nty;
    const int rr = tile / g.nty;
    const int txi = rr % g.ntx;
    const int tzi = rr / g.ntx;
    TileXYZ t;
    t.x0 = txi * g.BX * g.V;
    t.y0 = tyi * g.BY;
    t.z0 = tzi * g.ZC;
    return t;
}

template <typename T, int NF, int P>
__global__ void __launch_bounds__(256, 2) scalar_pass_kernel(const ScalarArgs A) {
    DevState* st = A.st;
    if (st->error) return;
    constexpr int V = VecT<T>::V;
    constexpr int NS = 6 * NF + 2;
    constexpr int NA = 2 * NF;
    constexpr int kFold = sizeof(T) == 4 ? 8 : 1 << 30;  // planes per FP32 run of the thread sums
    const Geometry& G = A.geo;
    const int N = G.N, BX = G.BX, BY = G.BY, ZC = G.ZC, S = G.S;
    const int TX = BX * V, RW = TX + 2 * V, ROWS = BY + 2;
    const int ASZ = ROWS * RW;  // elements of one array in one stage
    const int STG = NA * ASZ;   // elements of one stage
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw + 128);
    __shared__ double bacc[8][16];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int lin = ty * BX + tx;
    const int nthr = BX * BY;
    const int lane = lin & 31, warp = lin >> 5, nwarps = (nthr + 31) >> 5;
    const int nlanes = min(32, nthr - 32 * warp);
    const unsigned wmask = nlanes >= 32 ? 0xffffffffu : ((1u << nlanes) - 1u);
    for (int i = lin; i < 8 * 16; i += nthr) (&bacc[0][0])[i] = 0.0;

    const T cd = T(st->cd), A1 = T(st->A1), A3 = T(st->A3);
    const T h1 = T(A.pi.h1), h = T(A.pi.h), idx2 = T(A.mc.idx2);
    const T lam = T(A.mc.lam), q = T(A.mc.q);
    T fb[2], sf[2], sp[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        fb[f] = f < NF ? T(st->phibar[f]) : T(0);
        sf[f] = f < NF ? T(st->sphi[f]) : T(0);
        sp[f] = f < NF ? T(st->spi[f]) : T(0);
    }
    const T P0 = fb[0] * fb[0], C0 = fb[1] * fb[1];

    const int my_tiles = (blockIdx.x < (unsigned)G.ntiles) ? (G.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    // Load sequence of this block: for each of its tiles, planes z0-1 .. z0+ZC.  The
    // producer side walks it with counters (tile k, plane p, stage slot) so that no
    // division is needed per plane; the tile decode happens once per tile.
    int ld_k = 0, ld_p = 0, ld_slot = 0;
    TileXYZ ld_t = decode_tile(G, (int)blockIdx.x);
    const bool yhalo = (ty == 0) || (ty == BY - 1);
    const bool xhalo = (tx == 0) || (tx == BX - 1);
    const int yh_row = (ty == 0) ? 0 : BY + 1;
    const int xh_col = (tx == 0) ? V - 1 : V + TX;

    // Every thread copies its own part of the next load into its stage with cp.async:
    // its 16-byte vector of every array, the y-halo row vector (first/last thread row)
    // and the x-halo cell (first/last thread column), periodic indices.  One commit
    // group per load, empty past the end, so every thread counts groups alike.
    auto issue = [&]() {
        if (ld_k < my_tiles) {
            int z = ld_t.z0 - 1 + ld_p;
            z = z < 0 ? z + N : (z >= N ? z - N : z);
            T* dst = sm + ld_slot * STG;
            const int x = ld_t.x0 + tx * V, y = ld_t.y0 + ty;
            const size_t zoff = (size_t)z * N * N;
            const int yh = (ty == 0) ? (y == 0 ? N - 1 : y - 1) : (y == N - 1 ? 0 : y + 1);
            const int xh = (tx == 0) ? (x == 0 ? N - 1 : x - 1) : (x + V == N ? 0 : x + V);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const T* src = static_cast<const T*>(A.in[a]) + zoff;
                T* d = dst + a * ASZ;
                cp_async16(d + (ty + 1) * RW + V + tx * V, src + (size_t)y * N + x);
                if (yhalo) {
                    cp_async16(d + yh_row * RW + V + tx * V, src + (size_t)yh * N + x);
                    if (BY == 1) cp_async16(d + (BY + 1) * RW + V + tx * V, src + (size_t)(y == N - 1 ? 0 : y + 1) * N + x);
                }
                if (xhalo) {
                    cp_async_elem(d + (ty + 1) * RW + xh_col, src + (size_t)y * N + xh);
                    if (BX == 1) cp_async_elem(d + (ty + 1) * RW + V + TX, src + (size_t)y * N + (x + V == N ? 0 : x + V));
                }
            }
            if (++ld_p == ZC + 2) {
                ld_p = 0;
                if (++ld_k < my_tiles) ld_t = decode_tile(G, (int)blockIdx.x + ld_k * (int)gridDim.x);
            }
            if (++ld_slot == S) ld_slot = 0;
        }
        cp_async_commit();
    };
    // wait until load `need` has landed for every thread: `issued - 1 - need`
    // newer commit groups may stay pending
    int issued = 0;
    auto wait_for = [&](int need) {
        switch (issued - 1 - need) {
            case 0: cp_async_wait<0>(); break;
            case 1: cp_async_wait<1>(); break;
            case 2: cp_async_wait<2>(); break;
            case 3: cp_async_wait<3>(); break;
            case 4: cp_async_wait<4>(); break;
            default: cp_async_wait<5>(); break;
        }
        __syncthreads();
    };

    for (int L = 0; L < S; ++L, ++issued) issue();
    int sl_m = 0;   // stage slot of plane z-1; z and z+1 follow cyclically
    int need = 2;   // index of the load holding plane z+1

    // In-place drift of this thread's part of a landed stage: phi <- (phi - sphi) + cd (pi - spi)
    // for its own vector and the halo cells it copied, so that neighbours read drifted
    // values (each site is drifted once per pass).  Returns its own drifted vector and
    // shifted momentum.
    const T c0[2] = {sf[0] + cd * sp[0], sf[1] + cd * sp[1]};
    auto drift_stage = [&](T* Sx, T (&fo)[NF][V], T (&po)[NF][V]) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T* F = Sx + f * ASZ;
            const T* Pp = Sx + (NF + f) * ASZ;
            const int ob = (ty + 1) * RW + V + tx * V;
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
                if (BY == 1) {
                    const int ob2 = (BY + 1) * RW + V + tx * V;
                    vload_s(F + ob2, rf);
                    vload_s(Pp + ob2, rp);
#pragma unroll
                    for (int v = 0; v < V; ++v) rf[v] = (rf[v] + cd * rp[v]) - c0[f];
                    vstore(F + ob2, rf);
                }
            }
            if (xhalo) {
                const int oc = (ty + 1) * RW + xh_col;
                F[oc] = (F[oc] + cd * Pp[oc]) - c0[f];
                if (BX == 1) {
                    const int oc2 = (ty + 1) * RW + V + TX;
                    F[oc2] = (F[oc2] + cd * Pp[oc2]) - c0[f];
                }
            }
        }
    };

    for (int k = 0; k < my_tiles; ++k) {
        const TileXYZ tt = decode_tile(G, (int)blockIdx.x + k * (int)gridDim.x);
        const int x = tt.x0 + tx * V, y = tt.y0 + ty;
        const size_t NN = (size_t)N * N;
        const int ob = (ty + 1) * RW + V + tx * V;  // own vector inside an array block
        T ts[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) ts[i] = T(0);
        T fm[NF][V], fc[NF][V], fp[NF][V], pc[NF][V], pn[NF][V];
        // Runs of kFold planes: in FP32 the thread sums cover at most 4 kFold sites
        // before the warp folds them into its FP64 accumulators (FP64: one run per
        // tile).  FP32: unrolled by two, the register rotation of the z-queue
        // (fm <- fc <- fp) is renamed away in every other plane instead of moved
        // (FP64 keeps the loop rolled: unrolled it would spill).
        for (int zf = 0; zf < ZC; zf += kFold) {
            const int zend = ZC - zf < kFold ? ZC : zf + kFold;
#pragma unroll(sizeof(T) == 4 ? 2 : 1)
            for (int zz = zf; zz < zend; ++zz, ++need) {
                wait_for(need);  // planes z-1, z, z+1 have landed
                // the stage of plane z-2 was released by the previous iteration and every
                // thread has passed the barrier above: refill it now (one barrier per plane)
                if (zz > 0) { issue(); ++issued; }
                const int sl_c = sl_m + 1 == S ? 0 : sl_m + 1;
                const int sl_p = sl_c + 1 == S ? 0 : sl_c + 1;
                T* Sc = sm + sl_c * STG;
                T* Sp = sm + sl_p * STG;
                if (zz == 0) {
                    T* Sm = sm + sl_m * STG;
                    T dummy[NF][V];
                    drift_stage(Sm, fm, dummy);
                    drift_stage(Sc, fc, pc);
                }
                drift_stage(Sp, fp, pn);
                if (zz == 0) __syncthreads();  // halos of the tile's first plane are drifted
                T lap[NF][V];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T* cF = Sc + f * ASZ;
                    // x-neighbours: shuffles of the drifted own vectors, shared memory at row/warp edges
                    const T fromL = __shfl_up_sync(wmask, fc[f][V - 1], 1);
                    const T fromR = __shfl_down_sync(wmask, fc[f][0], 1);
                    const bool useL = (tx > 0) && (lane > 0), useR = (tx < BX - 1) && (lane < nlanes - 1);
                    const T left = useL ? fromL : cF[ob - 1];
                    const T right = useR ? fromR : cF[ob + V];
                    T u[V], d[V];
                    vload_s(cF + ob - RW, u);
                    vload_s(cF + ob + RW, d);
                    T g = T(0);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const T xl = (v == 0) ? left : fc[f][v - 1];
                        const T xr = (v == V - 1) ? right : fc[f][v + 1];
                        const T c = fc[f][v];
                        lap[f][v] = (((xl + xr) + (u[v] + d[v])) + (fm[f][v] + fp[f][v]) - T(6) * c) * idx2;
                        const T gx = xr - c, gy = d[v] - c, gz = fp[f][v] - c;
                        g += gx * gx + gy * gy + gz * gz;
                    }
                    ts[6 * f + 4] += g;
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
                if (A.write) {
                    const size_t o = (size_t)(tt.z0 + zz) * NN + (size_t)y * N + x;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        vstore_cs(static_cast<T*>(A.out[f]) + o, fc[f]);
                        vstore_cs(static_cast<T*>(A.out[NF + f]) + o, pout[f]);
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
            fold_warp_sums<T, NS>(ts, bacc[warp], lane, nlanes);
        }
        __syncthreads();  // the tile's last three stages are free
        issue();
        issue();
        issue();
        issued += 3;
        need += 2;
        sl_m = sl_m + 2 >= S ? sl_m + 2 - S : sl_m + 2;
    }
    cp_async_wait<0>();
    __syncthreads();

    // ---- block reduction (FP64) and last-block finish
    if (lin < NS) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += bacc[w][lin];
        A.partials[(size_t)blockIdx.x * NS + lin] = t;
    }
    __threadfence();
    __syncthreads();
    __shared__ unsigned int last;
    if (lin == 0) last = (atomicAdd(A.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // fixed-order compensated FP64 sum of the partials: warp w handles sums w, w+nwarps, ...
    __shared__ double tot[kMaxSums];
    const double invV = A.mc.inv_vol;
    for (int s = warp; s < NS; s += nwarps) {
        const double r = warp_partials_sum(A.partials, (int)gridDim.x, NS, s, lane, nlanes);
        if (lane == 0) tot[s] = r * invV;
    }
    __syncthreads();
    if (lin == 0) {
        *A.counter = 0u;
        scalar_finish(st, tot, A.mc, A.pi, sizeof(T) == 4);
    }
}

// In-place drift of the leapfrog closing step: delta_phi <- (delta_phi - sphi) + cd (delta_pi - spi).
template <typename T>
__global__ void scalar_drift_kernel(T* phi0, T* phi1, const T* pi0, const T* pi1, int nf, size_t n, DevState* st) {
    if (st->error) return;
    const T cd = T(st->cd);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int f = 0; f < nf; ++f) {
        T* ph = f == 0 ? phi0 : phi1;
        const T* pp = f == 0 ? pi0 : pi1;
        const T sf = T(st->sphi[f]), sp = T(st->spi[f]);
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
            ph[i] = (ph[i] - sf) + cd * (pp[i] - sp);
    }
}

// --------------------------------------------------------------- host side

template <typename T, int NF> static const void* kptr_p(int pexp) {
    if (pexp == 4) return (const void*)scalar_pass_kernel<T, NF, 4>;
    if (pexp == 6) return (const void*)scalar_pass_kernel<T, NF, 6>;
    return (const void*)scalar_pass_kernel<T, NF, 2>;
}

static const void* scalar_kernel_ptr(const Lattice* L) {
    if (L->prec == CL_FP32) return L->mc.nf == 1 ? kptr_p<float, 1>(L->mc.pexp) : kptr_p<float, 2>(L->mc.pexp);
    return L->mc.nf == 1 ? kptr_p<double, 1>(L->mc.pexp) : kptr_p<double, 2>(L->mc.pexp);
}

// Tile geometry.  CL_SCALAR_TILE="BY,ZC,S[,BX]" (rows per tile, planes per z
// chunk, ring stages, threads per row: 16, 32 or 64) overrides the defaults;
// values that do not fit N are ignored.
void scalar_geometry(Lattice* L) {
    Geometry& g = L->geo;
    int want_by = 8, want_zc = 128, want_s = 5, want_bx = 32;
    if (const char* env = getenv("CL_SCALAR_TILE")) {
        int a = 0, b = 0, c = 0, d = 0;
        const int got = sscanf(env, "%d,%d,%d,%d", &a, &b, &c, &d);
        if (got >= 3 && a > 0 && b > 0 && c >= 3 && c <= 8) {
            want_by = a;
            want_zc = b;
            want_s = c;
            if (got == 4 && (d == 16 || d == 32 || d == 64)) want_bx = d;
        }
    }
    const int N = L->mc.N;
    g.N = N;
    g.V = (L->prec == CL_FP32) ? 4 : 2;
    const int nv = N / g.V;
    int bx = nv < want_bx ? nv : want_bx;
    while (nv % bx != 0) --bx;
    g.BX = bx;
    int by = 256 / g.BX;
    if (g.BX == want_bx && want_by < by) by = want_by;
    if (by > N) by = N;
    while (N % by != 0) --by;
    g.BY = by;
    int zc = N < want_zc ? N : want_zc;
    while (N % zc != 0) --zc;
    // small lattices: shorter z columns, then fewer rows, until the tiles can
    // occupy every SM twice (a 32^3 lattice would otherwise be one tile)
    const int target = 2 * L->sm_count;
    auto count = [&](int byv, int zcv) { return (N / (g.BX * g.V)) * (N / byv) * (N / zcv); };
    while (count(g.BY, zc) < target && zc % 2 == 0 && zc / 2 >= 4) zc /= 2;
    while (count(g.BY, zc) < target && g.BY % 2 == 0 && g.BY / 2 >= 4 && g.BX * g.BY / 2 >= 64) g.BY /= 2;
    g.ZC = zc;
    g.ntx = N / (g.BX * g.V);
    g.nty = N / g.BY;
    g.ntz = N / g.ZC;
    g.ntiles = g.ntx * g.nty * g.ntz;
    g.threads = g.BX * g.BY;
    const size_t RW = (size_t)g.BX * g.V + 2 * g.V;
    const size_t stage = 2 * (size_t)L->mc.nf * (g.BY + 2) * RW * L->tsize;
    g.S = want_s;
    while (g.S > 4 && 128 + (size_t)g.S * stage > 227 * 1024) --g.S;
    g.smem = 128 + (size_t)g.S * stage;
    int per_sm = 1;
    const void* fn = scalar_kernel_ptr(L);
    // one attribute per kernel for all lattices: allow the largest ring the device
    // permits (opt-in limit minus the kernel's static shared memory)
    {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        cudaGetLastError();  // leave no error state behind
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g.threads, g.smem);
    if (per_sm < 1) per_sm = 1;
    int grid = L->sm_count * per_sm;
    if (grid > g.ntiles) grid = g.ntiles;
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    g.grid = grid;
}

template <typename T, int NF, int P>
static cudaError_t launch_t(Lattice* L, const ScalarArgs& A, cudaStream_t s) {
    const Geometry& g = L->geo;
    auto fn = scalar_pass_kernel<T, NF, P>;
    fn<<<g.grid, dim3(g.BX, g.BY), g.smem, s>>>(A);
    return cudaGetLastError();
}

template <typename T, int NF>
static cudaError_t launch_p(Lattice* L, const ScalarArgs& A, cudaStream_t s) {
    switch (L->mc.pexp) {
        case 2: return launch_t<T, NF, 2>(L, A, s);
        case 4: return launch_t<T, NF, 4>(L, A, s);
        case 6: return launch_t<T, NF, 6>(L, A, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t scalar_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s) {
    ScalarArgs A;
    const int nf = L->mc.nf;
    for (int i = 0; i < 4; ++i) { A.in[i] = nullptr; A.out[i] = nullptr; }
    for (int i = 0; i < 2 * nf; ++i) {
        A.in[i] = L->buf.f[src][i];
        A.out[i] = L->buf.f[dst][i];
    }
    A.st = L->buf.st;
    A.partials = L->buf.partials;
    A.counter = L->buf.counter;
    A.mc = L->mc;
    A.geo = L->geo;
    A.pi = pi;
    A.write = write ? 1 : 0;
    if (L->prec == CL_FP32) return nf == 1 ? launch_p<float, 1>(L, A, s) : launch_p<float, 2>(L, A, s);
    return nf == 1 ? launch_p<double, 1>(L, A, s) : launch_p<double, 2>(L, A, s);
}

cudaError_t scalar_launch_drift(Lattice* L, int cur, cudaStream_t s) {
    const size_t n = (size_t)L->mc.N * L->mc.N * L->mc.N;
    const int nf = L->mc.nf;
    void** b = L->buf.f[cur];
    const int grid = L->sm_count * 8;
    if (L->prec == CL_FP32)
        scalar_drift_kernel<float><<<grid, 256, 0, s>>>((float*)b[0], nf > 1 ? (float*)b[1] : nullptr,
                                                        (const float*)b[nf], nf > 1 ? (const float*)b[nf + 1] : nullptr,
                                                        nf, n, L->buf.st);
    else
        scalar_drift_kernel<double><<<grid, 256, 0, s>>>((double*)b[0], nf > 1 ? (double*)b[1] : nullptr,
                                                         (const double*)b[nf],
                                                         nf > 1 ? (const double*)b[nf + 1] : nullptr, nf, n, L->buf.st);
    return cudaGetLastError();
}

}  // namespace cl
