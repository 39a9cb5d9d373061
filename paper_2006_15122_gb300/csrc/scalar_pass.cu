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
// Tiling: a block of BX x BY threads owns a tile of TX = BX*V by BY sites in
// x-y (V = 4 floats or 2 doubles per thread, 16-byte accesses) and marches ZC
// planes in z; z-neighbours live in registers, x-y neighbours of the drifted
// plane in a ring of S shared-memory stages, one plane each (one barrier per
// plane).  Each plane arrives by tensor-memory-access copies (TMA) issued by
// up to four warps from the middle of the block, one array each: per array the
// interior box (TX x BY), the two halo rows (TX x 1) and the two halo column
// strips (V x BY), periodic wrap by the choice of each box's coordinates; one
// mbarrier per stage counts the bytes, and one other warp waits on it for the
// block.  Plane z+S-2 is requested while plane z is computed.  The grid is persistent
// (grid-stride over tiles, y-tiles fastest so that y-halos are L2 hits of
// concurrently running tiles).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "cl_internal.cuh"
#include "scalar_common.cuh"

namespace cl {

struct ScalarArgs {
    // tensor maps of the source arrays, [slot][box]: box 0 the tile interior
    // (TX x BY x 1), box 1 one row (TX x 1 x 1), box 2 one column strip (V x BY x 1)
    CUtensorMap tm[4][3];
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

// Byte layout of one array's block in a ring stage.  Every region starts on a
// 128-byte boundary (the alignment of a tensor copy's destination): the tile
// interior [BY][TX], the row y0-1 [TX] ("up"), the row y0+BY [TX] ("down"),
// the columns x0-V..x0-1 [BY][V] ("left") and x0+TX..x0+TX+V-1 [BY][V] ("right").
struct StageLayout {
    uint32_t up, down, left, right, arr;  // byte offsets in the block; arr: the block's size
};
__host__ __device__ __forceinline__ uint32_t round128(uint32_t b) { return (b + 127u) & ~127u; }
__host__ __device__ __forceinline__ StageLayout stage_layout(int BX, int BY, int V, int tsize) {
    const uint32_t row = (uint32_t)(BX * V * tsize), col = (uint32_t)(BY * V * tsize);
    StageLayout s;
    s.up = round128(row * (uint32_t)BY);
    s.down = s.up + round128(row);
    s.left = s.down + round128(row);
    s.right = s.left + round128(col);
    s.arr = s.right + round128(col);
    return s;
}

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

// FB = 8 or 16: the tile of 32 x FB threads is compiled in (32 x 8 is the shape
// of every lattice with N a multiple of 128 in FP32, 64 in FP64; 32 x 16 one
// 512-thread block per SM), so the stage layout and the neighbour offsets are
// constants; FB = 0: they come from the geometry (at most 256 threads).
template <typename T, int NF, int P, int FB>
__global__ void __launch_bounds__(FB == 16 ? 512 : 256, FB == 16 ? 1 : 2)
    scalar_pass_kernel(const __grid_constant__ ScalarArgs A) {
    constexpr bool FIXED = FB != 0;
    DevState* st = A.st;
    if (st->error) return;
    constexpr int V = VecT<T>::V;
    constexpr int NS = 6 * NF + 2;
    constexpr int NA = 2 * NF;
    constexpr int kFold = sizeof(T) == 4 ? 8 : 1 << 30;  // planes per FP32 run of the thread sums
    const Geometry& G = A.geo;
    const int N = G.N, BX = FIXED ? 32 : G.BX, BY = FIXED ? FB : G.BY, ZC = G.ZC, S = G.S;
    const int TX = BX * V;
    const StageLayout SL = stage_layout(BX, BY, V, (int)sizeof(T));
    const int AE = (int)(SL.arr / sizeof(T));  // elements of one array block
    const int STG = NA * AE;                   // elements of one stage
    const uint32_t plane_bytes = (uint32_t)(NA * sizeof(T)) * (uint32_t)(TX * BY + 2 * TX + 2 * BY * V);
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~(uintptr_t)127);
    const uint32_t sm_addr = smem_u32(sm);
    __shared__ double bacc[16][16];
    __shared__ __align__(8) uint64_t full[8];  // one per stage: the plane's bytes have landed
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int lin = ty * BX + tx;
    const int nthr = BX * BY;
    const int lane = FIXED ? tx : lin & 31, warp = FIXED ? ty : lin >> 5, nwarps = (nthr + 31) >> 5;
    const int nlanes = min(32, nthr - 32 * warp);
    const unsigned wmask = nlanes >= 32 ? 0xffffffffu : ((1u << nlanes) - 1u);
    for (int i = lin; i < 16 * 16; i += nthr) (&bacc[0][0])[i] = 0.0;
    // nprod producer warps issue the copies, producer pw those of arrays pw, pw + nprod, ...
    // They are taken from the middle of the block, away from the first and last
    // thread rows, which drift the y-halo rows.  Producer warps need five lanes:
    // blocks have at least 16 threads (N >= 8), and only the last warp can be partial.
    const int full5 = nwarps - (nthr - 32 * (nwarps - 1) < 5 ? 1 : 0);
    const int nprod = full5 < NA ? full5 : NA;
    const int pw = warp - (full5 - nprod) / 2;
    const bool producer = pw >= 0 && pw < nprod;
    if (lin == 0) {
        for (int i = 0; i < S; ++i) mbar_init(&full[i], (uint32_t)nprod);
        fence_mbar_init();
    }

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

    // This thread's vector and its four x-y neighbours inside an array block
    // (elements): interior rows, or the halo regions at the tile's edges.
    const int o_own = ty * TX + tx * V;
    const int o_u = ty > 0 ? o_own - TX : (int)(SL.up / sizeof(T)) + tx * V;
    const int o_d = ty < BY - 1 ? o_own + TX : (int)(SL.down / sizeof(T)) + tx * V;
    const int o_l = tx > 0 ? o_own - 1 : (int)(SL.left / sizeof(T)) + ty * V + (V - 1);
    const int o_r = tx < BX - 1 ? o_own + V : (int)(SL.right / sizeof(T)) + ty * V;

    // Load sequence of this block: for each of its tiles, planes z0-1 .. z0+ZC,
    // load i into stage i mod S.  Each producer warp walks it with counters (tile
    // k, plane p, stage slot); its lane 0 posts the byte count of its arrays on
    // the stage's mbarrier (one arrival per producer warp, before its copies),
    // and lanes 0-4 each copy one box kind of those arrays.
    int ld_k = 0, ld_p = 0, ld_slot = 0;
    int pending = 0;  // producer lanes: loads issued and not yet waited for
    TileXYZ ld_t = decode_tile(G, (int)blockIdx.x);
    const int my_arrays = producer ? (NA - 1 - pw) / nprod + 1 : 0;
    const uint32_t warp_bytes = plane_bytes / NA * (uint32_t)my_arrays;
    auto issue = [&]() {  // producer warps only
        if (ld_k >= my_tiles) return;
        int z = ld_t.z0 - 1 + ld_p;
        z = z < 0 ? z + N : (z >= N ? z - N : z);
        uint64_t* bar = &full[ld_slot];
        if (lane == 0) mbar_arrive_expect_tx(bar, warp_bytes);
        __syncwarp(wmask);
        if (lane < 5) {
            const int kind = lane, x0 = ld_t.x0, y0 = ld_t.y0;
            int cx = x0, cy = y0, box = 0;
            uint32_t off = 0;
            if (kind == 1) { cy = y0 == 0 ? N - 1 : y0 - 1; box = 1; off = SL.up; }
            if (kind == 2) { cy = y0 + BY == N ? 0 : y0 + BY; box = 1; off = SL.down; }
            if (kind == 3) { cx = x0 == 0 ? N - V : x0 - V; box = 2; off = SL.left; }
            if (kind == 4) { cx = x0 + TX == N ? 0 : x0 + TX; box = 2; off = SL.right; }
            const uint32_t dst = sm_addr + (uint32_t)ld_slot * (uint32_t)(STG * sizeof(T)) + off;
            for (int a = pw; a < NA; a += nprod) tma_load_3d(dst + (uint32_t)a * SL.arr, &A.tm[a][box], cx, cy, z, bar);
        }
        ++pending;
        if (++ld_p == ZC + 2) {
            ld_p = 0;
            if (++ld_k < my_tiles) ld_t = decode_tile(G, (int)blockIdx.x + ld_k * (int)gridDim.x);
        }
        if (++ld_slot == S) ld_slot = 0;
    };
    // Loads are taken in order (stage wslot, phase parity wpar).  One warp, the
    // poller (neither a producer nor a halo row), waits for them before the plane's
    // barrier, suspended in try_wait, so that only one warp spends issue slots on
    // waiting.  The completion of a tensor copy carries an implicit async-to-generic
    // proxy fence, the poller's wait acquires the completed phase, and the barrier
    // (release/acquire at CTA scope) orders that before every thread's reads of the
    // stage.  A wait that gives up sets `late`; the barrier makes the block leave its
    // tile loop together.
    const bool poller = warp == (nwarps > 2 ? nwarps - 2 : 0);
    int wslot = 0;
    uint32_t wpar = 0;
    bool late = false, failed = false;
    auto wait_loads = [&](int k) {  // poller, before the barrier
        int sl = wslot;
        uint32_t par = wpar;
        for (int i = 0; i < k; ++i) {
            if (!mbar_wait_bounded_sleep(&full[sl], par)) late = true;
            if (++sl == S) { sl = 0; par ^= 1u; }
        }
    };
    auto take_loads = [&](int k) {  // every thread, after the barrier
        for (int i = 0; i < k; ++i) {
            --pending;
            if (++wslot == S) { wslot = 0; wpar ^= 1u; }
        }
    };

    __syncthreads();  // barriers initialized
    if (producer)
        for (int L = 0; L < S; ++L) issue();
    int sl_m = 0;   // stage slot of plane z-1; z and z+1 follow cyclically

    // In-place drift of this thread's part of a landed stage: phi <- (phi - sphi) + cd (pi - spi)
    // for its own vector and the halo cells that it reads for its neighbours at the tile's
    // edges, so that neighbours read drifted values (each site is drifted once per pass).
    // Returns its own drifted vector and shifted momentum.
    const T c0[2] = {sf[0] + cd * sp[0], sf[1] + cd * sp[1]};
    auto drift_stage = [&](T* Sx, T (&fo)[NF][V], T (&po)[NF][V]) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T* F = Sx + f * AE;
            const T* Pp = Sx + (NF + f) * AE;
            T rf[V], rp[V];
            vload_s(F + o_own, rf);
            vload_s(Pp + o_own, rp);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                po[f][v] = rp[v] - sp[f];
                fo[f][v] = (rf[v] + cd * rp[v]) - c0[f];
            }
            vstore(F + o_own, fo[f]);
            if (ty == 0) {
                vload_s(F + o_u, rf);
                vload_s(Pp + o_u, rp);
#pragma unroll
                for (int v = 0; v < V; ++v) rf[v] = (rf[v] + cd * rp[v]) - c0[f];
                vstore(F + o_u, rf);
            }
            if (ty == BY - 1) {
                vload_s(F + o_d, rf);
                vload_s(Pp + o_d, rp);
#pragma unroll
                for (int v = 0; v < V; ++v) rf[v] = (rf[v] + cd * rp[v]) - c0[f];
                vstore(F + o_d, rf);
            }
            if (tx == 0) F[o_l] = (F[o_l] + cd * Pp[o_l]) - c0[f];
            if (tx == BX - 1) F[o_r] = (F[o_r] + cd * Pp[o_r]) - c0[f];
        }
    };

    for (int k = 0; k < my_tiles; ++k) {
        const TileXYZ tt = decode_tile(G, (int)blockIdx.x + k * (int)gridDim.x);
        const int x = tt.x0 + tx * V, y = tt.y0 + ty;
        const size_t NN = (size_t)N * N;
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
            for (int zz = zf; zz < zend; ++zz) {
                // planes z-1, z, z+1 have landed (z-1 and z were waited for earlier,
                // except at the tile's first plane)
                const int nload = zz == 0 ? 3 : 1;
                if (poller) wait_loads(nload);
                // Proxy fence: this thread's in-place drift writes (generic proxy) are
                // ordered before later tensor copies into the same stage (async proxy).
                // A stage written at plane z is refilled after the barrier of plane z+3
                // at the earliest (z+1 for the tile's first plane, z = 0), or at the
                // tile's end: a fence at every odd plane and one before the tile-end
                // barrier cover every case.
                if (zz & 1) fence_proxy_async_smem();
                if (__syncthreads_or(late)) {
                    failed = true;
                    goto drain;
                }
                take_loads(nload);
                // the stage of plane z-2 was released by the previous iteration and every
                // thread has passed the barrier above: refill it now (one barrier per plane)
                if (zz > 0 && producer) issue();
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
                    const T* cF = Sc + f * AE;
                    // x-neighbours: shuffles of the drifted own vectors, shared memory at row/warp edges
                    const T fromL = __shfl_up_sync(wmask, fc[f][V - 1], 1);
                    const T fromR = __shfl_down_sync(wmask, fc[f][0], 1);
                    const bool useL = (tx > 0) && (lane > 0), useR = (tx < BX - 1) && (lane < nlanes - 1);
                    const T left = useL ? fromL : cF[o_l];
                    const T right = useR ? fromR : cF[o_r];
                    T u[V], d[V];
                    vload_s(cF + o_u, u);
                    vload_s(cF + o_d, d);
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
        fence_proxy_async_smem();
        __syncthreads();  // the tile's last three stages are free
        if (producer) {
            issue();
            issue();
            issue();
        }
        sl_m = sl_m + 2 >= S ? sl_m + 2 - S : sl_m + 2;
    }
drain:
    if (failed) {
        // a plane never arrived (not expected): flag the pass, let the copies still
        // in flight land (each wait again bounded) before the block's memory is released
        if (lane == 0 && producer) {
            st->error = kErrCopyTimeout;
            int slot = wslot;
            uint32_t par = wpar;
            for (int i = 0; i < pending; ++i) {
                mbar_wait_bounded(&full[slot], par);
                if (++slot == S) { slot = 0; par ^= 1u; }
            }
        }
    }
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

// the compiled-in tile for this geometry: 8 or 16 rows of 32 threads, else 0
static int fixed_tile(const Geometry& g) { return g.BX == 32 && (g.BY == 8 || g.BY == 16) ? g.BY : 0; }

template <typename T, int NF, int FB> static const void* kptr_p(int pexp) {
    if (pexp == 4) return (const void*)scalar_pass_kernel<T, NF, 4, FB>;
    if (pexp == 6) return (const void*)scalar_pass_kernel<T, NF, 6, FB>;
    return (const void*)scalar_pass_kernel<T, NF, 2, FB>;
}
template <typename T, int NF> static const void* kptr_f(const Lattice* L) {
    const int fb = fixed_tile(L->geo);
    if constexpr (sizeof(T) == 4)  // the 32 x 16 tile exists in FP32 only
        if (fb == 16) return kptr_p<T, NF, 16>(L->mc.pexp);
    return fb == 8 ? kptr_p<T, NF, 8>(L->mc.pexp) : kptr_p<T, NF, 0>(L->mc.pexp);
}

static const void* scalar_kernel_ptr(const Lattice* L) {
    if (L->prec == CL_FP32) return L->mc.nf == 1 ? kptr_f<float, 1>(L) : kptr_f<float, 2>(L);
    return L->mc.nf == 1 ? kptr_f<double, 1>(L) : kptr_f<double, 2>(L);
}

// Tile geometry.  CL_SCALAR_TILE="BY,ZC,S[,BX]" (rows per tile, planes per z
// chunk, ring stages, threads per row: 16, 32 or 64) overrides the defaults;
// values that do not fit N are ignored.
void scalar_geometry(Lattice* L) {
    Geometry& g = L->geo;
    // FP32: 32 x 16 threads (one 512-thread block per SM, half the y-halo re-reads of 32 x 8); FP64: 32 x 8
    int want_by = L->prec == CL_FP32 ? 16 : 8, want_zc = 128, want_s = 5, want_bx = 32;
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
    // at most 256 threads, except the compiled-in 32 x 16 tile in FP32 (one 512-thread block per SM)
    int by = 256 / g.BX;
    if (g.BX == want_bx && want_by < by) by = want_by;
    if (g.BX == 32 && want_bx == 32 && want_by == 16 && L->prec == CL_FP32) by = 16;
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
    const size_t stage = 2 * (size_t)L->mc.nf * stage_layout(g.BX, g.BY, g.V, (int)L->tsize).arr;
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
    const int fb = fixed_tile(g);
    auto fn = fb == 8 ? scalar_pass_kernel<T, NF, P, 8> : scalar_pass_kernel<T, NF, P, 0>;
    if constexpr (sizeof(T) == 4)
        if (fb == 16) fn = scalar_pass_kernel<T, NF, P, 16>;
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

// The three tensor maps of one N^3 array (x fastest): the tile interior
// (TX x BY), one row (TX x 1) and one column strip (V x BY), one z plane each.
// Out-of-range parts of a box are never requested (halos wrap by coordinate).
static bool encode_array_maps(CUtensorMap (&tm)[3], const void* base, const Geometry& g, size_t tsize) {
    const int TX = g.BX * g.V;
    return encode_plane_box(&tm[0], base, g.N, tsize, TX, g.BY) && encode_plane_box(&tm[1], base, g.N, tsize, TX, 1) &&
           encode_plane_box(&tm[2], base, g.N, tsize, g.V, g.BY);
}

cudaError_t scalar_launch_pass(Lattice* L, int src, int dst, const PassInfo& pi, bool write, cudaStream_t s) {
    ScalarArgs A;
    memset(&A, 0, sizeof(A));
    const int nf = L->mc.nf;
    for (int i = 0; i < 2 * nf; ++i) {
        A.in[i] = L->buf.f[src][i];
        A.out[i] = L->buf.f[dst][i];
        if (!encode_array_maps(A.tm[i], A.in[i], L->geo, L->tsize)) return cudaErrorInvalidValue;
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
