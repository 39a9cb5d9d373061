// Shared-memory plane ring of the z-marching gauge passes (the SU(2) kick and
// the U(1) pass).
//
// A block of BX x BY threads, one site each, owns a BX x BY tile in x-y and
// marches a run of planes in z.  NA arrays of T are staged plane by plane with
// cp.async in a ring of S >= 4 stages: while plane z computes, planes z-1, z
// and z+1 are resident (each with a one-cell x-y halo, corners included) and
// the next plane is in flight, with one block barrier per plane.
//
// Stage layout: array a, row r (0 .. BY+1 for y0-1 .. y0+BY), column c, at
// a * ASZ + r * RW + c; the interior of a row starts at c = V (16-byte aligned,
// V = 16 / sizeof(T)), the x-halo cells sit at V-1 and V+BX.
//
// Work split: the (x-y tile, z) plane tiles, numbered x-y tile major with the
// y-tiles fastest, are cut into equal contiguous ranges, one per block; a
// segment is the part of a range inside one x-y tile, and loads its planes
// z0-1 .. z0+len (periodic).  Every thread of the block walks the same
// segments, so all barriers are block-uniform.
#pragma once

#include "cl_internal.cuh"

namespace cl {

template <typename T, int NA, int BX, int BY>
struct PlaneRing {
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int RW = BX + 2 * V, ROWS = BY + 2, ASZ = ROWS * RW, STG = NA * ASZ;
    static constexpr int NT = BX * BY;
    static constexpr int VPR = BX / V;      // 16-byte vectors per row
    static constexpr int VPA = ROWS * VPR;  // vectors per array and plane, y-halo rows included
    static constexpr int HPA = 2 * ROWS;    // x-halo cells per array and plane, corners included
    static_assert(BX % V == 0, "a tile row is a whole number of 16-byte vectors");

    struct Seg {
        int x0, y0, z0, len;
    };

    T* sm;
    const T* const* src;  // NA array bases (a table in shared memory)
    int N, S, nty, lin;
    long long beg, end;
    // loader: segment being loaded, plane within it, next stage slot
    long long ld_cur;
    Seg ls;
    int ld_p, ld_slot;
    // consumer: commit groups issued, load index of plane z+1, stage slot of plane z-1
    int issued, need, sl_m;

    // Bytes of dynamic shared memory for S stages (128 bytes of alignment slack).
    __host__ __device__ static size_t bytes(int stages) { return 128 + (size_t)stages * STG * sizeof(T); }
    // Plane tiles of an N^3 lattice.
    __host__ __device__ static long long plane_tiles(int n) { return (long long)(n / BX) * (n / BY) * n; }

    __device__ __forceinline__ Seg seg_at(long long cur) const {
        Seg g;
        const long long xy = cur / N;
        g.z0 = (int)(cur - xy * N);
        g.len = (int)min((long long)(N - g.z0), end - cur);
        g.y0 = (int)(xy % nty) * BY;
        g.x0 = (int)(xy / nty) * BX;
        return g;
    }

    // One commit group: the next plane of the load sequence (an empty group past the end).
    __device__ __forceinline__ void issue() {
        if (ld_cur < end) {
            int z = ls.z0 - 1 + ld_p;
            z = z < 0 ? z + N : (z >= N ? z - N : z);
            T* dst = sm + ld_slot * STG;
            const size_t zoff = (size_t)z * N * N;
#pragma unroll
            for (int e0 = 0; e0 < NA * VPA; e0 += NT) {
                const int e = e0 + lin;
                if (e < NA * VPA) {
                    const int a = e / VPA, r = (e % VPA) / VPR, v = e % VPR;
                    int y = ls.y0 - 1 + r;
                    y = y < 0 ? y + N : (y >= N ? y - N : y);
                    cp_async16(dst + a * ASZ + r * RW + V + v * V, src[a] + zoff + (size_t)y * N + ls.x0 + v * V);
                }
            }
#pragma unroll
            for (int e0 = 0; e0 < NA * HPA; e0 += NT) {
                const int e = e0 + lin;
                if (e < NA * HPA) {
                    const int a = e / HPA, side = (e % HPA) / ROWS, r = e % ROWS;
                    int y = ls.y0 - 1 + r;
                    y = y < 0 ? y + N : (y >= N ? y - N : y);
                    const int x = side == 0 ? (ls.x0 == 0 ? N - 1 : ls.x0 - 1) : (ls.x0 + BX == N ? 0 : ls.x0 + BX);
                    cp_async_elem(dst + a * ASZ + r * RW + (side == 0 ? V - 1 : V + BX),
                                  src[a] + zoff + (size_t)y * N + x);
                }
            }
            if (++ld_p == ls.len + 2) {
                ld_p = 0;
                ld_cur += ls.len;
                if (ld_cur < end) ls = seg_at(ld_cur);
            }
            if (++ld_slot == S) ld_slot = 0;
        }
        cp_async_commit();
        ++issued;
    }

    // Wait until load `need` has landed for every thread (issued - 1 - need newer
    // groups may stay in flight), then a block barrier.
    __device__ __forceinline__ void wait_need() {
        switch (issued - 1 - need) {
            case 0: cp_async_wait<0>(); break;
            case 1: cp_async_wait<1>(); break;
            case 2: cp_async_wait<2>(); break;
            case 3: cp_async_wait<3>(); break;
            case 4: cp_async_wait<4>(); break;
            default: cp_async_wait<5>(); break;
        }
        __syncthreads();
    }

    // Set up this block's range and put the first S loads in flight.  The caller
    // has made the source table visible to the block (a barrier after filling it).
    __device__ __forceinline__ void start(T* smem, const T* const* table, int n, int stages, int thread) {
        sm = smem;
        src = table;
        N = n;
        S = stages;
        lin = thread;
        nty = n / BY;
        const long long W = plane_tiles(n);
        beg = W * blockIdx.x / gridDim.x;
        end = W * (blockIdx.x + 1) / gridDim.x;
        ld_cur = beg;
        ls = seg_at(beg);
        ld_p = 0;
        ld_slot = 0;
        issued = 0;
        need = 2;
        sl_m = 0;
        for (int L = 0; L < S; ++L) issue();
    }

    // Plane zz of the current segment: after this, planes z-1, z, z+1 are resident;
    // the stage of plane z-2, free since the barrier, is refilled.
    __device__ __forceinline__ void begin_plane(int zz) {
        wait_need();
        if (zz > 0) issue();
    }
    // Stage of plane z + dz, dz = -1, 0, 1.
    __device__ __forceinline__ const T* stage(int dz) const {
        int s = sl_m + 1 + dz;
        s = s >= S ? s - S : s;
        return sm + s * STG;
    }
    __device__ __forceinline__ void end_plane() {
        sl_m = sl_m + 1 == S ? 0 : sl_m + 1;
        ++need;
    }
    // After the last plane of a segment: its three stages are free once every
    // thread is past the barrier; they take the next loads.
    __device__ __forceinline__ void end_segment() {
        __syncthreads();
        issue();
        issue();
        issue();
        need += 2;
        sl_m = sl_m + 2 >= S ? sl_m + 2 - S : sl_m + 2;
    }
    __device__ __forceinline__ void finish() { cp_async_wait<0>(); }
};

}  // namespace cl
