// The render's chunk of work (Sec. 3.1-3.4 for a range of rays, deposit into
// a shared-memory tile), shared by the render, batch and ray-list kernels,
// which live in their own translation units so that they compile in
// parallel.
#pragma once

#include "trace.cuh"

namespace pivbos {

constexpr int kRenderThreads = 256;
constexpr int kRenderMinBlocks = 4;   // CTAs per SM the register budget must allow
constexpr int kBatchMinBlocks = 3;    // ... for the persistent batch kernel (4 would spill 112 B)
// Work: the flattened (Morton slot, ray) index space (sources in Morton order,
// read as double-float from P.src_df) is cut into chunks of
// rays_per_cta consecutive rays; a CTA takes one chunk, so its rays come
// from one source or a few neighbouring ones and their spots fall in one
// 32x32 shared tile anchored at the first hit.
// Shared memory of one CTA working on one chunk of rays.
struct ChunkShared {
    unsigned long long tile[kTileW * kTileH];
    uint32_t order[kMaxOrderRays];
    unsigned long long cnt[PIVBOS_RAY_NSTATUS];
    int anchor_tid, ax, ay;
};

// Rays [first, last) of the flattened (Morton slot, ray) space of one render:
// trace (in mid-plane Morton order in dense media), deposit into the shared
// tile anchored at the first hit, flush the tile, add the status counts.
// Every thread of the CTA must call it; it leaves `sh` free for reuse.
template <int INTEG, bool CACHE, bool EXT>
__device__ __forceinline__ void render_chunk(const TraceParams& P, ChunkShared& sh, uint64_t first, uint64_t last,
                                             int64_t* __restrict__ image, int64_t* __restrict__ stats)
{
    for (int q = threadIdx.x; q < kTileW * kTileH; q += blockDim.x) sh.tile[q] = 0ull;
    if (threadIdx.x == 0) {
        sh.anchor_tid = 0x7fffffff;
        sh.ax = -(1 << 28);
        sh.ay = -(1 << 28);
    }
    if (threadIdx.x < PIVBOS_RAY_NSTATUS) sh.cnt[threadIdx.x] = 0ull;
    __syncthreads();

    const uint32_t rps = P.rays_per_source;
    unsigned cnt[PIVBOS_RAY_NSTATUS] = {0, 0, 0, 0, 0, 0};

    // In a dense medium, trace the CTA's rays in the order of where they
    // cross the box: a warp then gathers from a few neighbouring cells
    // instead of the whole cone of a source.
    const uint32_t n_here = (uint32_t)(last - first);
    const bool reorder = P.reorder && n_here <= (uint32_t)kMaxOrderRays;
    if (reorder) order_chunk(P, sh.order, first, n_here);
    // one uniform loop over the chunk's rays; after the first round every
    // thread's first hit is known and the lowest-thread hit anchors the tile
    const int rounds = (int)((n_here + blockDim.x - 1) / blockDim.x);
    int ax = -(1 << 28), ay = -(1 << 28);
    for (int round = 0; round < rounds; ++round) {
        const uint32_t e = (uint32_t)round * blockDim.x + threadIdx.x;
        const bool active = e < n_here;
        const uint64_t idx = first + (reorder && active ? (sh.order[e] & 0x7ffu) : e);
        RayOut r;
        r.status = PIVBOS_RAY_MISS;
        if (active) {
            const uint32_t flat = P.ray_list ? __ldg(P.ray_list + idx) : (uint32_t)idx;
            const uint32_t slot = flat / rps, k = flat - slot * rps;
            const uint32_t sid = __ldg(P.perm + slot) + P.source_offset;
            const float2* s = P.src_df + 3 * (size_t)slot;
            const float2 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2);
            trace_ray<INTEG, CACHE, EXT>(P, df{a.x, a.y}, df{b.x, b.y}, df{c.x, c.y}, sid, k, r, nullptr);
            cnt[r.status]++;
        }
        if (round == 0) {
            if (active && r.status == PIVBOS_RAY_REACHED) atomicMin(&sh.anchor_tid, (int)threadIdx.x);
            __syncthreads();
            if ((int)threadIdx.x == sh.anchor_tid) {
                float f;
                sh.ax = df_floor(r.px, f) - kTileW / 2;
                sh.ay = df_floor(r.py, f) - kTileH / 2;
            }
            __syncthreads();
            ax = sh.ax;
            ay = sh.ay;
        }
        // every lane of the warp reaches this ballot (the loop is uniform)
        const unsigned dep = __ballot_sync(0xffffffffu, active && r.status == PIVBOS_RAY_REACHED);
        if (active && r.status == PIVBOS_RAY_REACHED) {
            if constexpr (EXT) deposit_ray<true>(P.o, r.px, r.py, sh.tile, ax, ay, image, r.w, dep);
            else deposit_ray(P.o, r.px, r.py, sh.tile, ax, ay, image, 1.0f, dep);
        }
    }
    if (stats) {
#pragma unroll
        for (int q = 0; q < PIVBOS_RAY_NSTATUS; ++q) {
            unsigned v = cnt[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(&sh.cnt[q], (unsigned long long)v);
        }
    }
    __syncthreads();
    // flush the tile: one global atomic per touched pixel
    for (int q = threadIdx.x; q < kTileW * kTileH; q += blockDim.x) {
        const unsigned long long v = sh.tile[q];
        if (v) {
            const int gx = ax + (q % kTileW), gy = ay + (q / kTileW);
            atomicAdd(reinterpret_cast<unsigned long long*>(&image[(size_t)gy * P.o.W + gx]), v);
        }
    }
    if (stats && threadIdx.x < PIVBOS_RAY_NSTATUS && sh.cnt[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[threadIdx.x]), sh.cnt[threadIdx.x]);
    __syncthreads();
}

}  // namespace pivbos
