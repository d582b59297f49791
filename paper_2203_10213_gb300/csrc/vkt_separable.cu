// vkt_separable.cu -- ApplyFilter for a rank-1 filter w[c][b][a] = gz[c] gy[b] gx[a]
// (the Gaussian blur of Sec. 4.3 is one), as three fused 1-D passes.
//
// The clamp-to-edge correlation factorises per axis, so the 3-D result equals an x pass,
// then a y pass, then a z pass, each clamped at its own faces.  One CTA owns a TX x TY
// column and marches through a chunk of z.  Per input plane: TMA brings the raw tile
// (with halo), it is converted to float with clamping, the x pass writes (TY+2r) x TX
// partial sums to shared memory, the y pass reduces them to this thread's RY x RX block
// in registers, and the z pass adds gz[c] times that block into the K output planes the
// input plane touches (K x RY x RX accumulators per thread).  HBM traffic is the source
// once plus the destination once; 3k FMAs per voxel.
#include <algorithm>
#include <cstdio>

#include "vkt_internal.h"
#include "vkt_tile.cuh"

namespace vkt {
namespace {

constexpr int NT = 256;
constexpr int BX = 16, BY = 16;
constexpr int RX = 4, RY = 2;
constexpr int TX = BX * RX, TY = BY * RY;
constexpr int STAGES = 4;

template <int K>
struct SepW {
    float gx[K], gy[K], gz[K];
};

struct SepArgs {
    const void* src;
    void* dst;
    int nx, ny, nz;
    int sfmt, dfmt;
    int zchunk;
    int use_tma;
    float a0, a1, qmax;
    unsigned* status;
};

template <int K>
__host__ __device__ constexpr size_t sep_smem_bytes(int sfmt)
{
    using Geo = Brick<K, TX, TY>;
    return 128 + static_cast<size_t>(STAGES) * Geo::raw_bytes(sfmt) +
           static_cast<size_t>(Geo::FH) * Geo::FP * sizeof(float) +      // float tile
           static_cast<size_t>(Geo::FH) * TX * sizeof(float);            // x-pass output
}

template <int K>
__global__ void __launch_bounds__(NT)
    k_separable(const __grid_constant__ CUtensorMap tmap, const SepArgs p, const SepW<K> G)
{
    using Geo = Brick<K, TX, TY>;
    constexpr int R = Geo::R, FH = Geo::FH, FP = Geo::FP;
    constexpr int XGROUPS = TX / 4;                     // x-pass items per row
    constexpr int XITEMS = FH * XGROUPS;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    const int rawb = Geo::raw_bytes(p.sfmt);
    const uint32_t txb = Geo::raw_tx(p.sfmt);
    unsigned char* raw = smem + 128;
    float* F = reinterpret_cast<float*>(raw + STAGES * rawb);
    float* T1 = F + FH * FP;

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zc0 = blockIdx.z * p.zchunk;
    const int zc1 = min(zc0 + p.zchunk, p.nz);
    if (zc0 >= zc1) return;
    const int pfirst = zc0 - R;
    const int nplanes = zc1 - zc0 + 2 * R;
    const int xa = fmt_xalign(p.sfmt);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        if (p.use_tma) prefetch_tensor_map(&tmap);
    }
    __syncthreads();
    int issued = 0;
    if (p.use_tma && tid == 0) {
        for (int s = 0; s < STAGES && s < nplanes; ++s, ++issued) {
            mbar_arrive_expect_tx(&bars[s], txb);
            tma_load_3d(raw + s * rawb, &tmap, &bars[s], x0 - xa, y0 - R,
                        clampi(pfirst + s, 0, p.nz - 1));
        }
    }

    ConvPlan<Geo, NT> plan;
    plan.init(p.sfmt, p.nx, p.ny, x0, y0, tid);

    float acc[K][RY][RX];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int x = 0; x < RX; ++x) acc[s][i][x] = 0.f;

    const int ox = x0 + tx * RX;
    const int nvalid = p.nx - ox;
    bool failed = false;

    auto plane = [&](const int it, const int u) {
        const int s = it % STAGES;
        const unsigned char* rs = raw + s * rawb;
        bool ok = true;
        if (p.use_tma) {
            ok = mbar_wait(&bars[s], (it / STAGES) & 1);
        } else {
            fill_raw_plain<Geo, NT>(const_cast<unsigned char*>(rs), p.src, p.sfmt, p.nx, p.ny,
                                    x0, y0, clampi(pfirst + it, 0, p.nz - 1), tid);
            __syncthreads();
        }
        if (ok) plan.convert(rs, p.sfmt, F, tid);
        if (__syncthreads_or(!ok)) {
            failed = true;
            return;
        }
        if (p.use_tma && tid == 0 && it + STAGES < nplanes) {
            mbar_arrive_expect_tx(&bars[s], txb);
            tma_load_3d(raw + s * rawb, &tmap, &bars[s], x0 - xa, y0 - R,
                        clampi(pfirst + it + STAGES, 0, p.nz - 1));
            ++issued;
        }
        // x pass: T1[row][x] = sum_a gx[a] F[row][x + a], 4 outputs per item
#pragma unroll
        for (int n = 0; n < (XITEMS + NT - 1) / NT; ++n) {
            const int item = tid + n * NT;
            if (item < XITEMS) {
                const int row = item / XGROUPS, g = item - row * XGROUPS;
                float win[4 + K - 1];
                load_row<4 + K - 1, 4>(F + row * FP + 4 * g, win);
                float4 o;
                float* op = &o.x;
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    float t = 0.f;
#pragma unroll
                    for (int a = 0; a < K; ++a) t = fmaf(G.gx[a], win[x + a], t);
                    op[x] = t;
                }
                *reinterpret_cast<float4*>(T1 + row * TX + 4 * g) = o;
            }
        }
        __syncthreads();
        // y pass into registers, then the z pass into the K rotating accumulator planes
        float t2[RY][RX];
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int x = 0; x < RX; ++x) t2[i][x] = 0.f;
#pragma unroll
        for (int j = 0; j < RY + K - 1; ++j) {
            float v[RX];
            load_row<RX, RX>(T1 + (ty * RY + j) * TX + tx * RX, v);
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const int b = j - i;
                if (b < 0 || b >= K) continue;
#pragma unroll
                for (int x = 0; x < RX; ++x) t2[i][x] = fmaf(G.gy[b], v[x], t2[i][x]);
            }
        }
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const int sl = ((u - c + R) % K + K) % K;
#pragma unroll
            for (int i = 0; i < RY; ++i)
#pragma unroll
                for (int x = 0; x < RX; ++x) acc[sl][i][x] = fmaf(G.gz[c], t2[i][x], acc[sl][i][x]);
        }
        const int sl0 = ((u - R) % K + K) % K;
        if (it >= 2 * R) {
            const int oz = pfirst + it - R;
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const int oy = y0 + ty * RY + i;
                if (oy < p.ny && nvalid > 0) {
                    const int64_t idx = (static_cast<int64_t>(oz) * p.ny + oy) * p.nx + ox;
                    store_row<RX>(p.dst, p.dfmt, idx, nvalid, acc[sl0][i], p.a0, p.a1, p.qmax);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int x = 0; x < RX; ++x) acc[sl0][i][x] = 0.f;
    };

    for (int g = 0; g * K < nplanes && !failed; ++g) {
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int it = g * K + u;
            if (it >= nplanes || failed) break;
            plane(it, u);
        }
    }

    if (failed) {
        if (tid == 0) {
            atomicOr(p.status, STATUS_TIMEOUT);
            for (int it = issued - 1; it >= 0 && it >= issued - STAGES; --it)
                mbar_wait(&bars[it % STAGES], (it / STAGES) & 1);
        }
        __syncthreads();
    }
}

template <int K>
vktError launch_k(const Job& job, const float* gx, const float* gy, const float* gz,
                  const Ctx& ctx)
{
    using Geo = Brick<K, TX, TY>;
    SepArgs a;
    a.src = job.src;
    a.dst = job.dst;
    a.nx = job.nx;
    a.ny = job.ny;
    a.nz = job.nz;
    a.sfmt = job.sfmt;
    a.dfmt = job.dfmt;
    a.a0 = job.a0;
    a.a1 = job.a1;
    a.qmax = job.qmax;
    a.status = ctx.status;
    SepW<K> G;
    for (int i = 0; i < K; ++i) {
        G.gx[i] = gx[i];
        G.gy[i] = gy[i];
        G.gz[i] = gz[i];
    }
    const int bx = (job.nx + TX - 1) / TX;
    const int by = (job.ny + TY - 1) / TY;
    int sms = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const long target = static_cast<long>(sms) * 8;
    const long xy = static_cast<long>(bx) * by;
    int chunks = static_cast<int>(std::min<long>((target + xy - 1) / xy, std::max(1, job.nz / 8)));
    chunks = std::max(chunks, 1);
    a.zchunk = (job.nz + chunks - 1) / chunks;
    const int bz = (job.nz + a.zchunk - 1) / a.zchunk;

    alignas(64) CUtensorMap map;
    a.use_tma = encode_tensor_map_3d(&map, job.sfmt, job.src, job.nx, job.ny, job.nz,
                                     Geo::raw_w(job.sfmt), Geo::FH, 1)
                    ? 1
                    : 0;
    if (!a.use_tma) memset(&map, 0, sizeof(map));
    const size_t smem = sep_smem_bytes<K>(job.sfmt);
    cudaError_t e = cudaFuncSetAttribute(k_separable<K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return from_cuda(e);
    if (ctx.debug)
        fprintf(stderr, "[vkt] separable k=%d grid=(%d,%d,%d) zchunk=%d smem=%zu tma=%d\n", K,
                bx, by, bz, a.zchunk, smem, a.use_tma);
    k_separable<K><<<dim3(bx, by, bz), NT, smem, ctx.stream>>>(map, a, G);
    count_launches(1);
    return from_cuda(cudaGetLastError());
}

}  // namespace

vktError launch_separable(const Job& job, const float* gx, const float* gy, const float* gz,
                          int k, const Ctx& ctx)
{
    switch (k) {
    case 1: return launch_k<1>(job, gx, gy, gz, ctx);
    case 3: return launch_k<3>(job, gx, gy, gz, ctx);
    case 5: return launch_k<5>(job, gx, gy, gz, ctx);
    case 7: return launch_k<7>(job, gx, gy, gz, ctx);
    case 9: return launch_k<9>(job, gx, gy, gz, ctx);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

}  // namespace vkt
