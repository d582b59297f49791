// vkt_separable.cuh -- the single-volume separable kernels and their launcher, one
// instantiation per filter size k in its own translation unit (vkt_separable.cu: k = 1, 3
// and the dispatch; vkt_separable5/7/9.cu), so the unrolled kernels compile in parallel.
#pragma once

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "vkt_sep_brick.cuh"

namespace vkt {
namespace sepk {

// CTAs per SM the register allocation must allow: three up to k = 5 (the float32 and
// run-time-format kernels fit in 80 registers there), two for k = 7 and for the uint8
// kernels, whose fused word-load x pass needs about 120
template <int K, int SF>
constexpr int sep_min_blocks() { return (K <= 5 && SF != FMT_U8) ? 3 : 2; }

// planes in flight of a single-volume kernel: k for whole-volume tensor-map kernels up to
// k = 7, a ring whose stage and phase are compile-time constants of the k-times unrolled
// plane loop (measured 1 % faster than three stages at k = 5), else the batch brick's three
template <int K, int LM, bool ROI>
constexpr int ns_of() { return (LM == sep::LM_TMA && !ROI && K >= 3 && K <= 7) ? K : sep::FSTAGES; }

// SF/DF: source and destination formats fixed at compile time (-1: read from the job);
// LM: the way stages are filled (sep::LM_*), fixed at compile time where known
template <int K, int SF = -1, int DF = -1, int LM = sep::LM_ANY, bool ROI = false>
__global__ void __launch_bounds__(sep::NT, sep_min_blocks<K, SF>())
    k_separable(const __grid_constant__ CUtensorMap tmap, const sep::Job J, const sep::W<K> G,
                unsigned* status)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (threadIdx.x == 0) {
        sep::init_barriers(smem);
        if (LM != sep::LM_ROWS && J.use_tma) prefetch_tensor_map(&tmap);
    }
    __syncthreads();
    grid_dependency_wait();   // programmatic launch: the previous kernel's writes are visible
    launch_dependents();
    uint32_t gplane = 0;   // this CTA's only brick: the static ring applies when NS == K
    constexpr int NS = ns_of<K, LM, ROI>();
    sep::brick<K, sep::W<K>, SF, DF, LM, ROI, NS, NS == K>(J, G, &tmap, blockIdx.x, blockIdx.y,
                                                           blockIdx.z, smem, gplane, status);
}

template <int K, int LM = sep::LM_ANY, bool ROI = false>
__global__ void __launch_bounds__(sep::NT)
    k_separable_comp(const __grid_constant__ CUtensorMap tmap, const sep::Job J,
                     const sep::W<K> G, unsigned* status)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (threadIdx.x == 0) {
        sep::init_barriers(smem);
        if (LM != sep::LM_ROWS && J.use_tma) prefetch_tensor_map(&tmap);
    }
    __syncthreads();
    grid_dependency_wait();   // programmatic launch: the previous kernel's writes are visible
    launch_dependents();
    uint32_t gplane = 0;
    sep::brick_comp<K, sep::W<K>, LM, ROI>(J, G, &tmap, blockIdx.x, blockIdx.y, blockIdx.z, smem,
                                           gplane, status);
}

// the kernel for a job: tensor-map jobs and (for the compiled-in formats) row-copy jobs get
// kernels without the other ways of loading; plain-load jobs take the run-time variant
template <int K, int SF, int DF>
auto pick_fast(const sep::Job& J)
{
    if constexpr (SF >= 0) {
        if (J.use_tma) return k_separable<K, SF, DF, sep::LM_TMA>;
        if (J.rows) return k_separable<K, SF, DF, sep::LM_ROWS>;
        return k_separable<K, -1, -1, sep::LM_ANY>;
    } else {
        if (J.use_tma) return k_separable<K, -1, -1, sep::LM_TMA>;
        return k_separable<K, -1, -1, sep::LM_ANY>;
    }
}

template <int K>
vktError launch_k(const Job& job, const float* gx, const float* gy, const float* gz,
                  const Ctx& ctx)
{
    using Geo = Brick<K, sep::TX, sep::TY>;
    sep::Job J;
    memset(&J, 0, sizeof(J));
    J.src = job.src;
    J.dst = job.dst;
    J.nx = job.nx;
    J.ny = job.ny;
    J.nz = job.nz;
    J.sfmt = job.sfmt;
    J.dfmt = job.dfmt;
    J.k = K;
    J.a0 = job.a0;
    J.a1 = job.a1;
    J.qmax = job.qmax;
    J.comp = job.comp;
    J.a0lo = job.a0lo;
    J.a1lo = job.a1lo;
    // output region; the brick grid starts at a 16-byte boundary left of it (tensor-map
    // boxes start there) and stores only inside it
    int rx0, ry0, rz0, rx1, ry1, rz1;
    job_region(job, rx0, ry0, rz0, rx1, ry1, rz1);
    J.ox0 = rx0 - rx0 % fmt_xalign(job.sfmt);
    J.oy0 = ry0;
    J.oz0 = rz0;
    J.sx0 = rx0;
    J.sx1 = rx1;
    J.sy1 = ry1;
    J.sz1 = rz1;
    const int ex = rx1 - J.ox0, ey = ry1 - ry0, ez = rz1 - rz0;
    const int ty = J.comp ? sep::CTY : sep::TY;
    sep::W<K> G;
    for (int i = 0; i < K; ++i) {
        G.gx[i] = gx[i];
        G.gy[i] = gy[i];
        G.gz[i] = gz[i];
    }
    const int sms = ctx.sms;
    J.tiles_x = (ex + sep::TX - 1) / sep::TX;
    J.tiles_y = (ey + ty - 1) / ty;

    alignas(64) CUtensorMap map;
    J.use_tma = encode_tensor_map_3d(&map, job.sfmt, job.src, job.nx, job.ny, job.nz,
                                     Geo::raw_w(job.sfmt), ty + 2 * Geo::R, 1)
                    ? 1
                    : 0;
    // rows that no tensor map can describe are still fetched asynchronously, one bulk copy
    // per row, when the volume starts on a 16-byte boundary
    J.rows = (!J.use_tma && reinterpret_cast<uintptr_t>(J.src) % 16 == 0) ? 1 : 0;
    if (!J.use_tma) memset(&map, 0, sizeof(map));
    size_t smem = J.comp ? sep::smem_bytes_comp<K>(job.sfmt, J.rows != 0)
                         : sep::smem_bytes<K>(job.sfmt, J.rows != 0);
    // the common float32 destinations get kernels with their formats compiled in
    auto fast = pick_fast<K, -1, -1>(J);
    if constexpr (K >= 3 && K <= 7) {
        if (!J.comp && J.dfmt == FMT_F32 && J.sfmt == FMT_U8) fast = pick_fast<K, FMT_U8, FMT_F32>(J);
        if (!J.comp && J.dfmt == FMT_F32 && J.sfmt == FMT_F32) fast = pick_fast<K, FMT_F32, FMT_F32>(J);
    }
    auto comp = J.use_tma ? k_separable_comp<K, sep::LM_TMA> : k_separable_comp<K, sep::LM_ANY>;
    if (job.roi) {
        // region calls take variants that read the region fields: with the formats compiled
        // in for tensor-map jobs of the common float32 destinations, else run-time ones
        fast = k_separable<K, -1, -1, sep::LM_ANY, true>;
        comp = k_separable_comp<K, sep::LM_ANY, true>;
        if constexpr (K >= 3 && K <= 7) {
            if (!J.comp && J.use_tma && J.dfmt == FMT_F32 && J.sfmt == FMT_U8)
                fast = k_separable<K, FMT_U8, FMT_F32, sep::LM_TMA, true>;
            if (!J.comp && J.use_tma && J.dfmt == FMT_F32 && J.sfmt == FMT_F32)
                fast = k_separable<K, FMT_F32, FMT_F32, sep::LM_TMA, true>;
        }
    }
    // the tensor-map kernels of the compiled-in formats fuse the conversion into the x pass
    // (their own shared-memory layout)
    if (!J.comp && J.use_tma && J.dfmt == FMT_F32 &&
        (J.sfmt == FMT_F32 || J.sfmt == FMT_U8) && K >= 3 && K <= 7)
        smem = std::max(smem, sep::smem_bytes_fx<K, K>(job.sfmt));
    if (!J.comp && J.use_tma && !job.roi && K >= 3 && K <= 7)
        smem = std::max(smem, sep::smem_bytes<K, K>(job.sfmt, false));
    // z chunks sized for whole waves of the CTAs the chosen kernel keeps resident
    int per_sm = 1;
    vktError ve = prepare_kernel(ctx, J.comp ? reinterpret_cast<const void*>(comp)
                                             : reinterpret_cast<const void*>(fast),
                                 sep::NT, smem, &per_sm);
    if (ve != VKT_NO_ERROR) return ve;
    cudaError_t e = cudaSuccess;
    J.zchunk = job.zchunk > 0 ? std::min(job.zchunk, ez)
                             : zchunk_waves(static_cast<long>(J.tiles_x) * J.tiles_y, ez,
                                                  static_cast<long>(sms) * std::max(per_sm, 1), Geo::R);
    J.chunks = (ez + J.zchunk - 1) / J.zchunk;
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] separable%s k=%d grid=(%d,%d,%d) zchunk=%d smem=%zu tma=%d rows=%d\n",
                J.comp ? "-compensated" : "", K, J.tiles_x, J.tiles_y, J.chunks, J.zchunk, smem,
                J.use_tma, J.rows);
    const dim3 grid(J.tiles_x, J.tiles_y, J.chunks);
    e = J.comp ? launch_pdl(comp, grid, dim3(sep::NT), smem, ctx.stream, map, J, G, ctx.status)
               : launch_pdl(fast, grid, dim3(sep::NT), smem, ctx.stream, map, J, G, ctx.status);
    count_launches(1);
    if (e != cudaSuccess) return from_cuda(e);
    return from_cuda(cudaGetLastError());
}

}  // namespace sepk

// one launcher per filter size, defined in the translation unit of that size
vktError launch_separable_k1(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx);
vktError launch_separable_k3(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx);
vktError launch_separable_k5(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx);
vktError launch_separable_k7(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx);
vktError launch_separable_k9(const Job& job, const float* gx, const float* gy, const float* gz, const Ctx& ctx);

}  // namespace vkt
