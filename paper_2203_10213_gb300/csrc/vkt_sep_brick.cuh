// vkt_sep_brick.cuh -- one brick of the fused separable filter (three 1-D passes), shared by
// the single-volume kernel (vkt_separable.cu) and the batched persistent kernel
// (vkt_batch.cu).
//
// The clamp-to-edge correlation with w[c][b][a] = gz[c] gy[b] gx[a] factorises per axis,
// so it equals an x pass, then a y pass, then a z pass, each clamped at its own faces.  A
// brick is a TX x TY column of outputs over a chunk of z.  Per input plane: TMA brings the
// raw tile (with halo) into a ring of stages, it is converted to float with clamping, the
// x pass writes (TY+2r) x TX partial sums to shared memory, the y pass reduces them to the
// thread's RY x RX block in registers, and the z pass adds gz[c] times that block into the
// K output planes the input plane touches (K x RY x RX register accumulators); one output
// plane completes per input plane.  HBM traffic: the source once, the destination once.
#pragma once

#include "vkt_internal.h"
#include "vkt_tile.cuh"

namespace vkt {
namespace sep {

constexpr int NT = 256;
constexpr int BX = 16, BY = 16;
constexpr int RX = 4, RY = 2;
constexpr int TX = BX * RX, TY = BY * RY;
constexpr int CRY = 1;              // output rows per thread of the compensated brick
constexpr int CTY = BY * CRY;
constexpr int STAGES = 4;    // barriers per CTA; planes in flight of the compensated brick
constexpr int FSTAGES = 3;   // planes in flight of the float brick (measured faster than 4)
// How a brick fills its stages, fixed at compile time where the caller knows it (the plane
// loop is unrolled k times, so code for unused ways costs instruction cache):
// LM_ANY reads the job's use_tma / rows flags (else plain loads), LM_TMA and LM_ROWS assume one.
enum : int { LM_ANY = 0, LM_TMA = 1, LM_ROWS = 2 };
// the y and z passes run as packed two-lane FMAs over output pairs (x, x+1) for k <= 5 (at
// k >= 7, and in the run-time-format kernels at k = 5, the register pairs cost spills or
// more than the halved FMA issue saves); SF: the compile-time source format or -1
template <int K, int SF>
constexpr bool pair_yz() { return K <= 3 || (K == 5 && SF >= 0); }

// Everything a brick needs about its volume (the batched kernel reads these from a table).
struct Job {
    const void* src;
    void* dst;
    int nx, ny, nz;
    int sfmt, dfmt;
    int zchunk;
    int use_tma;
    int rows;          // no tensor map: stages filled by per-row bulk copies (issue_rows)
    // output region: bricks start at (ox0, oy0, oz0) and store the voxels with x in
    // [sx0, sx1), y < sy1, z < sz1 (the whole volume: set_whole_volume)
    int ox0, oy0, oz0;
    int sx0, sx1, sy1, sz1;
    int k;
    int tiles_x, tiles_y, chunks;
    float a0, a1, qmax;
    float g[3][VKT_MAX_FILTER_SIZE];    // x, y, z vectors
    // compensated mode (integer destinations): epilogue constants as double-float pairs
    int comp;
    float a0lo, a1lo;
};

inline void set_whole_volume(Job& J)
{
    J.ox0 = J.oy0 = J.oz0 = 0;
    J.sx0 = 0;
    J.sx1 = J.nx;
    J.sy1 = J.ny;
    J.sz1 = J.nz;
}

template <int K>
struct W {
    float gx[K], gy[K], gz[K];
};

// FX: the x pass reads the raw tensor-map stage directly (converting as it loads) into one of
// two x-pass tiles, so a plane needs one CTA barrier instead of two, no float tile, and none
// of the float tile's shared-memory traffic (about 14 of the 30 bytes per output voxel).  For
// float32 sources with tensor-map loads (17-21 % faster at k = 3, 5) and for uint8 sources,
// whose window is read as three aligned 32-bit words and converted with a byte permute
// (byte_float) instead of one byte load and one conversion per voxel (k = 5 on 512^3:
// 0.209 -> 0.199 ms at two CTAs per SM; at three it spills)
template <int LM, int SF, int K>
__host__ __device__ constexpr bool fused_x()
{
    return LM == LM_TMA && (SF == FMT_F32 || SF == FMT_U8);
}

// byte i (0..3) of word w as the float it codes (exact): 2^23 + code built by a byte permute,
// minus 2^23
__device__ __forceinline__ float byte_float(uint32_t w, int i)
{
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u + i)) - 8388608.f;
}

// the output tile of a brick with BXG threads along x (64 x 32 by default, 32 x 32 narrow)
// and of its compensated twin (64 x 16, 32 x 32 narrow)
template <int BXG>
constexpr int tile_x() { return BXG * RX; }
template <int BXG>
constexpr int tile_y() { return (NT / BXG) * (BXG == BX ? RY : 1); }
template <int BXG>
constexpr int tile_y_comp() { return (NT / BXG) * CRY; }

template <int K, int NS = FSTAGES, int BXG = BX>
__host__ __device__ constexpr size_t smem_bytes_fx(int sfmt)
{
    using Geo = Brick<K, tile_x<BXG>(), tile_y<BXG>()>;
    return 128 + static_cast<size_t>(NS) * Geo::stage_bytes(sfmt, false) +
           2 * static_cast<size_t>(Geo::FH) * tile_x<BXG>() * sizeof(float);
}

template <int K, int NS = FSTAGES, int BXG = BX>
__host__ __device__ constexpr size_t smem_bytes(int sfmt, bool rows = false)
{
    using Geo = Brick<K, tile_x<BXG>(), tile_y<BXG>()>;
    return 128 + static_cast<size_t>(NS) * Geo::stage_bytes(sfmt, rows) +
           static_cast<size_t>(Geo::FH) * Geo::FP * sizeof(float) +      // float tile
           static_cast<size_t>(Geo::FH) * tile_x<BXG>() * sizeof(float);  // x-pass output
}

// Initialises the stage barriers (thread 0; the caller synchronises afterwards).
__device__ __forceinline__ void init_barriers(unsigned char* smem)
{
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    for (int s = 0; s < 9; ++s) mbar_init(&bars[s], 1);   // up to 9 stages (in the 128-byte header)
    fence_mbar_init();
}

// Runs brick (bx, by, bz) of job J.  `gplane` counts the planes this CTA has brought in by
// TMA so far: stage = gplane % FSTAGES, parity = (gplane / FSTAGES) & 1, so the ring and its
// barrier phases carry on across bricks.  Returns false if a bounded wait timed out (after recording it and
// draining the loads in flight).
// ROI: the job's region fields (origin, store bounds) are read; otherwise the whole volume is
// assumed at compile time (no region arithmetic in the store path)
// ROTZ: the z pass keeps its K accumulator slots in a fixed order (the output plane an input
// plane reaches through tap c in slot K-1-c, slot 0 completing) and shifts them down after
// each plane, with one plane body in the loop; otherwise the loop is unrolled K times and the
// slots are compile-time rotations.  The unrolled form avoids the shifts and serves the
// single-volume kernels; the batch's persistent kernels (runtime formats, much code per
// plane) take ROTZ for K >= 5, where the unrolled body overflowed the instruction cache
// (256-volume batch: 1.354 -> 1.269 ms).
// NS: planes in flight (stages of the ring).  STATIC: the caller guarantees that this brick
// is the CTA's only one (gplane == 0 on entry: the single-volume kernels) and NS == K, so
// plane g*K + u of the K-times unrolled loop uses stage u and phase g, both known without
// arithmetic.  A persistent CTA (the batch) carries gplane from brick to brick and must use
// the general ring, whatever NS and K are.
template <int K, class Wt, int SF = -1, int DF = -1, int LM = LM_ANY, bool ROI = false,
          int NS = FSTAGES, bool STATIC = false, bool ROTZ = false, int BXG = BX>
__device__ __forceinline__ bool brick(const Job& J, const Wt& G, const CUtensorMap* tmap, int bx,
                                      int by, int bz, unsigned char* smem, uint32_t& gplane,
                                      unsigned* status)
{
    static_assert(!STATIC || NS == K, "the static ring has one stage per unrolled plane");
    // every launch of a brick has NT threads: the compiler may drop the bounds checks of the
    // per-thread item loops that this implies (3 % at k = 5 on 512^3)
    __builtin_assume(threadIdx.x < NT);
    // the brick's shape (shadowing the namespace's defaults): BXG threads along x, four
    // outputs each; the narrow shape (BXG = 8) has 32 x 32 outputs, one row per thread
    constexpr int BX = BXG, BY = NT / BXG;
    constexpr int RY = BXG == sep::BX ? sep::RY : 1;
    constexpr int TX = BX * RX, TY = BY * RY;
    using Geo = Brick<K, TX, TY>;
    constexpr int R = Geo::R, FH = Geo::FH, FP = Geo::FP;
    constexpr int XGROUPS = TX / 4;
    constexpr int XITEMS = FH * XGROUPS;

    // formats fixed at compile time (SF, DF >= 0) fold the format branches away
    const int sfmt = SF >= 0 ? SF : J.sfmt;
    const int dfmt = DF >= 0 ? DF : J.dfmt;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    const bool tma = LM == LM_TMA || (LM == LM_ANY && J.use_tma);
    const bool rows = LM == LM_ROWS || (LM == LM_ANY && J.rows);
    const int rawb = Geo::stage_bytes(sfmt, rows);
    const uint32_t txb = Geo::raw_tx(sfmt);
    unsigned char* raw = smem + 128;
    constexpr bool FX = fused_x<LM, SF, K>();
    float* F = reinterpret_cast<float*>(raw + NS * rawb);
    float* T1 = FX ? F : F + FH * FP;     // FX: two x-pass tiles, no float tile

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int x0 = (ROI ? J.ox0 : 0) + bx * TX, y0 = (ROI ? J.oy0 : 0) + by * TY;
    const int zc0 = (ROI ? J.oz0 : 0) + bz * J.zchunk;
    const int zc1 = min(zc0 + J.zchunk, ROI ? J.sz1 : J.nz);
    if (zc0 >= zc1) return true;
    const int pfirst = zc0 - R;
    const int nplanes = zc1 - zc0 + 2 * R;
    const int xa = fmt_xalign(sfmt);
    const uint32_t g0 = gplane;

    int issued = 0;
    const uint64_t vol_bytes =
        static_cast<uint64_t>(J.nx) * J.ny * J.nz * fmt_bytes(sfmt);
    if (tma && tid == 0) {
        for (int s = 0; s < NS && s < nplanes; ++s, ++issued) {
            const uint32_t q = g0 + s;
            mbar_arrive_expect_tx(&bars[q % NS], txb);
            tma_load_3d(raw + (q % NS) * rawb, tmap, &bars[q % NS], x0 - xa, y0 - R,
                        clampi(pfirst + s, 0, J.nz - 1));
        }
    } else if (rows) {
        for (int s = 0; s < NS && s < nplanes; ++s) {
            const uint32_t q = g0 + s;
            issue_rows<Geo, NT>(raw + (q % NS) * rawb, &bars[q % NS], J.src, vol_bytes,
                                sfmt, J.nx, J.ny, J.nz, x0, y0, pfirst + s, tid);
        }
        __syncthreads();   // every thread's expect_tx precedes the single arrival
        if (tid == 0)
            for (int s = 0; s < NS && s < nplanes; ++s, ++issued) mbar_arrive(&bars[(g0 + s) % NS]);
    }

    ConvPlan<Geo, NT> plan;
    plan.init(sfmt, J.nx, J.ny, x0, y0, tid, rows);

    // accumulators of the K output planes.  Packed kernels pair outputs (x, x+1) in one
    // float2, start at zero once, and afterwards give a slot's first tap in its z-march
    // (c = 0) as a plain product, so a retired slot needs no reset; the others keep scalar
    // accumulators that are reset after each store (fewer register-pair constraints)
    constexpr bool PAIR = pair_yz<K, SF>();
    float2 acc2[PAIR ? K : 1][RY][RX / 2];
    float acc[PAIR ? 1 : K][RY][RX];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int x = 0; x < RX; ++x) {
                if constexpr (PAIR) {
                    if (x % 2 == 0) acc2[s][i][x / 2] = make_float2(0.f, 0.f);
                } else {
                    acc[s][i][x] = 0.f;
                }
            }

    const int ox = x0 + tx * RX;
    const int nvalid = (ROI ? J.sx1 : J.nx) - ox;
    const int first = (ROI && J.sx0 > ox) ? J.sx0 - ox : 0;   // leading columns outside the region
    const int yend = ROI ? J.sy1 : J.ny;
    bool failed = false;

    auto plane = [&](const int it, const int u, const int gg) {
        const uint32_t q = g0 + it;
        const int s = STATIC ? u : static_cast<int>(q % NS);
        const uint32_t par = STATIC ? static_cast<uint32_t>(gg & 1) : ((q / NS) & 1);
        const unsigned char* rs = raw + s * rawb;
        bool ok = true;
        if constexpr (FX) {
            float* T1b = T1 + (it & 1) * FH * TX;
            ok = mbar_wait(&bars[s], par);
            // x pass straight from the raw stage: T1b[row][x] = sum_a gx[a] v(x + a - r), the
            // source voxels converted as they are loaded, clamped in x only at the volume's
            // x faces (the rows are clamped through the stage row read)
            constexpr int RWE = TX + 2 * fmt_xalign(SF);   // raw row length in voxels
            const bool xin = x0 - R >= 0 && x0 + TX - 1 + R <= J.nx - 1;
            if (ok) {
#pragma unroll
                for (int n = 0; n < (XITEMS + NT - 1) / NT; ++n) {
                    const int item = tid + n * NT;
                    if (item < XITEMS) {
                        const int row = item / XGROUPS, g = item - row * XGROUPS;
                        const int rrow = clampi(y0 - R + row, 0, J.ny - 1) - (y0 - R);
                        float win[4 + K - 1];
                        if constexpr (SF == FMT_U8) {
                            const unsigned char* rp = rs + rrow * RWE;
                            if (xin) {
                                // the item's K + 3 bytes start at raw column 4g + xa - R
                                // (xa = 16): the three aligned words from word g + W0 cover them
                                constexpr int W0 = (16 - R) / 4, O = (16 - R) & 3;
                                static_assert(O + K + 3 <= 12, "three words hold the window");
                                const uint32_t* wp = reinterpret_cast<const uint32_t*>(rp) + g + W0;
                                const uint32_t wd[3] = {wp[0], wp[1], wp[2]};
#pragma unroll
                                for (int e = 0; e < 4 + K - 1; ++e)
                                    win[e] = byte_float(wd[(O + e) >> 2], (O + e) & 3);
                            } else {
#pragma unroll
                                for (int e = 0; e < 4 + K - 1; ++e)
                                    win[e] = static_cast<float>(
                                        rp[clampi(x0 + 4 * g - R + e, 0, J.nx - 1) - (x0 - xa)]);
                            }
                        } else {
                            const float* rp = reinterpret_cast<const float*>(rs) + rrow * RWE;
                            if (xin) {
#pragma unroll
                                for (int e = 0; e < 4 + K - 1; ++e) win[e] = rp[4 * g - R + xa + e];
                            } else {
#pragma unroll
                                for (int e = 0; e < 4 + K - 1; ++e)
                                    win[e] = rp[clampi(x0 + 4 * g - R + e, 0, J.nx - 1) - (x0 - xa)];
                            }
                        }
                        float4 o;
                        float* op = &o.x;
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            float t = 0.f;
#pragma unroll
                            for (int a = 0; a < K; ++a) t = fmaf(G.gx[a], win[x + a], t);
                            op[x] = t;
                        }
                        *reinterpret_cast<float4*>(T1b + row * TX + 4 * g) = o;
                    }
                }
            }
            // the stage is read and the x-pass tile written by every thread
            if (__syncthreads_or(!ok)) {
                failed = true;
                return;
            }
            if (tid == 0 && it + NS < nplanes) {
                mbar_arrive_expect_tx(&bars[s], txb);
                tma_load_3d(raw + s * rawb, tmap, &bars[s], x0 - xa, y0 - R,
                            clampi(pfirst + it + NS, 0, J.nz - 1));
                ++issued;
            }
        } else {
        if (tma || rows) {
            ok = mbar_wait(&bars[s], par);
        } else {
            fill_raw_plain<Geo, NT>(const_cast<unsigned char*>(rs), J.src, sfmt, J.nx, J.ny,
                                    J.nz, x0, y0, pfirst + it, tid);
            __syncthreads();
        }
        if (ok) {
            if (rows) {
                const uint32_t zterm = static_cast<uint32_t>(clampi(pfirst + it, 0, J.nz - 1)) *
                                       static_cast<uint32_t>(J.ny) * static_cast<uint32_t>(J.nx);
                plan.convert_rows(rs, sfmt, F, tid, J.nx, J.ny, x0, y0, zterm);
            } else {
                plan.convert(rs, sfmt, F, tid);
            }
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            return;
        }
        if (tma && tid == 0 && it + NS < nplanes) {
            mbar_arrive_expect_tx(&bars[s], txb);
            tma_load_3d(raw + s * rawb, tmap, &bars[s], x0 - xa, y0 - R,
                        clampi(pfirst + it + NS, 0, J.nz - 1));
            ++issued;
        } else if (rows && it + NS < nplanes) {
            // all threads; the arrival follows the x-pass barrier below
            issue_rows<Geo, NT>(raw + s * rawb, &bars[s], J.src, vol_bytes, sfmt, J.nx, J.ny,
                                J.nz, x0, y0, pfirst + it + NS, tid);
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
        // the stage refilled by row copies above is complete in expectation: one arrival
        if (rows && tid == 0 && it + NS < nplanes) {
            mbar_arrive(&bars[s]);
            ++issued;
        }
        }   // not FX
        const float* T1y = FX ? T1 + (it & 1) * FH * TX : T1;
        // y pass into registers, then the z pass into the K rotating accumulator planes
        const int sl0 = ROTZ ? 0 : ((u - R) % K + K) % K;
        // stores the completed output plane it - R (once it >= 2R)
        auto store_plane = [&](const float (&rowv)[RX], int i) {
            const int oy = y0 + ty * RY + i;
            if (it >= 2 * R && oy < yend && nvalid > 0) {
                const int64_t idx = (static_cast<int64_t>(pfirst + it - R) * J.ny + oy) * J.nx + ox;
                store_row<RX>(J.dst, dfmt, idx, nvalid, rowv, J.a0, J.a1, J.qmax, first);
            }
        };
        if constexpr (PAIR) {
            float2 t2[RY][RX / 2];   // first tap of a row (b = 0) is a plain product
#pragma unroll
            for (int j = 0; j < RY + K - 1; ++j) {
                float v[RX];
                load_row<RX, RX>(T1y + (ty * RY + j) * TX + tx * RX, v);
#pragma unroll
                for (int i = 0; i < RY; ++i) {
                    const int b = j - i;
                    if (b < 0 || b >= K) continue;
                    const float2 w2 = make_float2(G.gy[b], G.gy[b]);
#pragma unroll
                    for (int x = 0; x < RX; x += 2) {
                        const float2 v2 = make_float2(v[x], v[x + 1]);
                        float2& d = t2[i][x >> 1];
                        d = (b == 0) ? __fmul2_rn(w2, v2) : __ffma2_rn(w2, v2, d);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const int sl = ROTZ ? K - 1 - c : ((u - c + R) % K + K) % K;
                const float2 w2 = make_float2(G.gz[c], G.gz[c]);
#pragma unroll
                for (int i = 0; i < RY; ++i)
#pragma unroll
                    for (int x = 0; x < RX / 2; ++x) {
                        float2& d = acc2[sl][i][x];
                        d = (c == 0) ? __fmul2_rn(w2, t2[i][x]) : __ffma2_rn(w2, t2[i][x], d);
                    }
            }
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                float rowv[RX];
#pragma unroll
                for (int x = 0; x < RX; x += 2) {
                    rowv[x] = acc2[sl0][i][x >> 1].x;
                    rowv[x + 1] = acc2[sl0][i][x >> 1].y;
                }
                store_plane(rowv, i);
            }
        } else {
            float t2[RY][RX];
#pragma unroll
            for (int i = 0; i < RY; ++i)
#pragma unroll
                for (int x = 0; x < RX; ++x) t2[i][x] = 0.f;
#pragma unroll
            for (int j = 0; j < RY + K - 1; ++j) {
                float v[RX];
                load_row<RX, RX>(T1y + (ty * RY + j) * TX + tx * RX, v);
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
                const int sl = ROTZ ? K - 1 - c : ((u - c + R) % K + K) % K;
#pragma unroll
                for (int i = 0; i < RY; ++i)
#pragma unroll
                    for (int x = 0; x < RX; ++x)
                        acc[sl][i][x] = fmaf(G.gz[c], t2[i][x], acc[sl][i][x]);
            }
#pragma unroll
            for (int i = 0; i < RY; ++i) store_plane(acc[sl0][i], i);
#pragma unroll
            for (int i = 0; i < RY; ++i)
#pragma unroll
                for (int x = 0; x < RX; ++x) acc[sl0][i][x] = 0.f;
        }
        if constexpr (ROTZ) {
#pragma unroll
            for (int q = 0; q + 1 < K; ++q)
#pragma unroll
                for (int i = 0; i < RY; ++i)
#pragma unroll
                    for (int x = 0; x < RX; ++x) {
                        if constexpr (PAIR) {
                            if (x % 2 == 0) acc2[q][i][x / 2] = acc2[q + 1][i][x / 2];
                        } else {
                            acc[q][i][x] = acc[q + 1][i][x];
                        }
                    }
            if constexpr (!PAIR) {
#pragma unroll
                for (int i = 0; i < RY; ++i)
#pragma unroll
                    for (int x = 0; x < RX; ++x) acc[K - 1][i][x] = 0.f;
            }
        }
    };

    if constexpr (ROTZ) {
#pragma unroll 1
        for (int it = 0; it < nplanes && !failed; ++it) plane(it, 0, 0);
    } else {
    for (int g = 0; g * K < nplanes && !failed; ++g) {
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int it = g * K + u;
            if (it >= nplanes || failed) break;
            plane(it, u, g);
        }
    }
    }
    // only bricks loaded through the stage barriers move them through their phases
    if (tma || rows) gplane = g0 + nplanes;

    if (failed) {
        if (tid == 0) {
            atomicOr(status, STATUS_TIMEOUT);
            for (int it = issued - 1; it >= 0 && it >= issued - NS; --it)
                mbar_wait(&bars[(g0 + it) % NS], ((g0 + it) / NS) & 1);
        }
        __syncthreads();
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------------------
// Compensated variant for integer destinations.  An FP32 sum of k taps per pass leaves an
// error of ~1e-2 of a 16-bit code, more than the 1e-3 LSB within which a rounding tie may
// go either way, so every pass carries a double-float (hi, lo) value built from the
// error-free transformations of vkt_tile.cuh (dot2_step, comp_code: the compensated dot
// product Dot2 of Ogita, Rump and Oishi), and the epilogue takes the rounding decision on
// the pair.  One output row per thread (RY = 1) keeps the 2 x k x 4 accumulators in
// registers.


template <int K, int BXG = BX>
__host__ __device__ constexpr size_t smem_bytes_comp(int sfmt, bool rows = false)
{
    using Geo = Brick<K, tile_x<BXG>(), tile_y_comp<BXG>()>;
    return 128 + static_cast<size_t>(STAGES) * Geo::stage_bytes(sfmt, rows) +
           static_cast<size_t>(Geo::FH) * Geo::FP * sizeof(float) +
           static_cast<size_t>(Geo::FH) * tile_x<BXG>() * sizeof(float2);  // (hi, lo) x pass
}

template <int K, class Wt, int LM = LM_ANY, bool ROI = false, int BXG = BX>
__device__ __forceinline__ bool brick_comp(const Job& J, const Wt& G, const CUtensorMap* tmap,
                                           int bx, int by, int bz, unsigned char* smem,
                                           uint32_t& gplane, unsigned* status)
{
    // the brick's shape (shadowing the namespace's defaults): BXG threads along x
    constexpr int BX = BXG, BY = NT / BXG;
    constexpr int TX = BX * RX, CTY = BY * CRY;
    __builtin_assume(threadIdx.x < NT);   // every launch of a brick has NT threads
    using Geo = Brick<K, TX, CTY>;
    constexpr int R = Geo::R, FH = Geo::FH, FP = Geo::FP;
    constexpr int XGROUPS = TX / 4;
    constexpr int XITEMS = FH * XGROUPS;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    const bool tma = LM == LM_TMA || (LM == LM_ANY && J.use_tma);
    const bool rows = LM == LM_ROWS || (LM == LM_ANY && J.rows);
    const int rawb = Geo::stage_bytes(J.sfmt, rows);
    const uint32_t txb = Geo::raw_tx(J.sfmt);
    unsigned char* raw = smem + 128;
    float* F = reinterpret_cast<float*>(raw + STAGES * rawb);
    float2* T1 = reinterpret_cast<float2*>(F + FH * FP);

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int x0 = (ROI ? J.ox0 : 0) + bx * TX, y0 = (ROI ? J.oy0 : 0) + by * CTY;
    const int zc0 = (ROI ? J.oz0 : 0) + bz * J.zchunk;
    const int zc1 = min(zc0 + J.zchunk, ROI ? J.sz1 : J.nz);
    if (zc0 >= zc1) return true;
    const int pfirst = zc0 - R;
    const int nplanes = zc1 - zc0 + 2 * R;
    const int xa = fmt_xalign(J.sfmt);
    const uint32_t g0 = gplane;

    int issued = 0;
    const uint64_t vol_bytes =
        static_cast<uint64_t>(J.nx) * J.ny * J.nz * fmt_bytes(J.sfmt);
    if (tma && tid == 0) {
        for (int s = 0; s < STAGES && s < nplanes; ++s, ++issued) {
            const uint32_t q = g0 + s;
            mbar_arrive_expect_tx(&bars[q % STAGES], txb);
            tma_load_3d(raw + (q % STAGES) * rawb, tmap, &bars[q % STAGES], x0 - xa, y0 - R,
                        clampi(pfirst + s, 0, J.nz - 1));
        }
    } else if (rows) {
        for (int s = 0; s < STAGES && s < nplanes; ++s) {
            const uint32_t q = g0 + s;
            issue_rows<Geo, NT>(raw + (q % STAGES) * rawb, &bars[q % STAGES], J.src, vol_bytes,
                                J.sfmt, J.nx, J.ny, J.nz, x0, y0, pfirst + s, tid);
        }
        __syncthreads();   // every thread's expect_tx precedes the single arrival
        if (tid == 0)
            for (int s = 0; s < STAGES && s < nplanes; ++s, ++issued) mbar_arrive(&bars[(g0 + s) % STAGES]);
    }
    ConvPlan<Geo, NT> plan;
    plan.init(J.sfmt, J.nx, J.ny, x0, y0, tid, rows);

    float acc_s[K][RX], acc_c[K][RX];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int x = 0; x < RX; ++x) acc_s[s][x] = acc_c[s][x] = 0.f;

    const int ox = x0 + tx * RX;
    const int oy = y0 + ty;
    const int nvalid = (ROI ? J.sx1 : J.nx) - ox;
    const int first = (ROI && J.sx0 > ox) ? J.sx0 - ox : 0;   // leading columns outside the region
    const int yend = ROI ? J.sy1 : J.ny;
    bool failed = false;

    auto plane = [&](const int it) {
        const uint32_t q = g0 + it;
        const int s = q % STAGES;
        const unsigned char* rs = raw + s * rawb;
        bool ok = true;
        if (tma || rows) {
            ok = mbar_wait(&bars[s], (q / STAGES) & 1);
        } else {
            fill_raw_plain<Geo, NT>(const_cast<unsigned char*>(rs), J.src, J.sfmt, J.nx, J.ny,
                                    J.nz, x0, y0, pfirst + it, tid);
            __syncthreads();
        }
        if (ok) {
            if (rows) {
                const uint32_t zterm = static_cast<uint32_t>(clampi(pfirst + it, 0, J.nz - 1)) *
                                       static_cast<uint32_t>(J.ny) * static_cast<uint32_t>(J.nx);
                plan.convert_rows(rs, J.sfmt, F, tid, J.nx, J.ny, x0, y0, zterm);
            } else {
                plan.convert(rs, J.sfmt, F, tid);
            }
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            return;
        }
        if (tma && tid == 0 && it + STAGES < nplanes) {
            mbar_arrive_expect_tx(&bars[s], txb);
            tma_load_3d(raw + s * rawb, tmap, &bars[s], x0 - xa, y0 - R,
                        clampi(pfirst + it + STAGES, 0, J.nz - 1));
            ++issued;
        } else if (rows && it + STAGES < nplanes) {
            // all threads; the arrival follows the x-pass barrier below
            issue_rows<Geo, NT>(raw + s * rawb, &bars[s], J.src, vol_bytes, J.sfmt, J.nx, J.ny,
                                J.nz, x0, y0, pfirst + it + STAGES, tid);
        }
        // x pass (inputs exact): T1[row][x] = Dot2(gx, F[row][x .. x+k-1])
#pragma unroll
        for (int n = 0; n < (XITEMS + NT - 1) / NT; ++n) {
            const int item = tid + n * NT;
            if (item < XITEMS) {
                const int row = item / XGROUPS, g = item - row * XGROUPS;
                float win[4 + K - 1];
                load_row<4 + K - 1, 4>(F + row * FP + 4 * g, win);
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    float hs, hc;
                    dot2_first_exact(G.gx[0], win[x], hs, hc);
#pragma unroll
                    for (int a = 1; a < K; ++a) dot2_exact(G.gx[a], win[x + a], hs, hc);
                    T1[row * TX + 4 * g + x] = make_float2(hs, hc);
                }
            }
        }
        __syncthreads();
        // the stage refilled by row copies above is complete in expectation: one arrival
        if (rows && tid == 0 && it + STAGES < nplanes) {
            mbar_arrive(&bars[s]);
            ++issued;
        }
        // y pass on the (hi, lo) pairs, then the z pass into the K rotating pair accumulators
        float ts[RX], tc[RX];
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const float2* r = T1 + (ty + b) * TX + tx * RX;
#pragma unroll
            for (int x = 0; x < RX; ++x) {
                const float2 v = r[x];
                if (b == 0)
                    dot2_first(G.gy[b], v.x, v.y, ts[x], tc[x]);
                else
                    dot2_step(G.gy[b], v.x, v.y, ts[x], tc[x]);
            }
        }
        // z pass: slot K-1-c holds the output plane that this input plane reaches through
        // tap c, so slot 0 completes now; the slots then shift down by one
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const int sl = K - 1 - c;
            // slot K-1 starts a new output plane: its first term sets it (no reset needed)
#pragma unroll
            for (int x = 0; x < RX; ++x) {
                if (c == 0)
                    dot2_first(G.gz[c], ts[x], tc[x], acc_s[sl][x], acc_c[sl][x]);
                else
                    dot2_step(G.gz[c], ts[x], tc[x], acc_s[sl][x], acc_c[sl][x]);
            }
        }
        constexpr int sl0 = 0;
        if (it >= 2 * R && oy < yend && nvalid > 0) {
            const int oz = pfirst + it - R;
            const int64_t idx = (static_cast<int64_t>(oz) * J.ny + oy) * J.nx + ox;
#pragma unroll
            for (int x = 0; x < RX; ++x) {
                if (x >= first && x < nvalid) {
                    const unsigned code = comp_code(acc_s[sl0][x], acc_c[sl0][x], J.a0, J.a0lo,
                                                    J.a1, J.a1lo, J.qmax);
                    if (J.dfmt == FMT_U16)
                        reinterpret_cast<uint16_t*>(J.dst)[idx + x] = static_cast<uint16_t>(code);
                    else
                        reinterpret_cast<unsigned char*>(J.dst)[idx + x] = static_cast<unsigned char>(code);
                }
            }
        }
#pragma unroll
        for (int q = 0; q + 1 < K; ++q)
#pragma unroll
            for (int x = 0; x < RX; ++x) {
                acc_s[q][x] = acc_s[q + 1][x];
                acc_c[q][x] = acc_c[q + 1][x];
            }
    };

    // one plane body, not unrolled: the Dot2 arithmetic of a plane is large, and a loop
    // unrolled k times (compile-time slots) overflowed the instruction cache (k = 7: the
    // batch's compensated kernel stalled on instruction fetch more than on anything else)
#pragma unroll 1
    for (int it = 0; it < nplanes && !failed; ++it) plane(it);
    if (tma || rows) gplane = g0 + nplanes;
    if (failed) {
        if (tid == 0) {
            atomicOr(status, STATUS_TIMEOUT);
            for (int it = issued - 1; it >= 0 && it >= issued - STAGES; --it)
                mbar_wait(&bars[(g0 + it) % STAGES], ((g0 + it) / STAGES) & 1);
        }
        __syncthreads();
        return false;
    }
    return true;
}

}  // namespace sep
}  // namespace vkt
