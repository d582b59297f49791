// vkt_direct.cuh -- direct FP32 evaluation of ApplyFilter (Sec. 3.2, "Volume Manipulation":
// a user-specified convolution kernel applied to every cell), all k^3 taps on CUDA cores.
// The kernel template and its launcher are instantiated by vkt_direct.cu (float
// accumulation, and the adjoint) and vkt_direct_comp.cu (compensated accumulation).
//
// Each CTA owns a TX x TY column of output voxels and marches through a chunk of z.  Input
// planes (with an r-voxel halo) arrive by TMA into a ring of raw tiles, are converted to
// float with clamp-to-edge into a float tile, and every input plane is multiplied into the
// K output planes it touches; each thread keeps K x RY x RX accumulators in registers, so
// an input plane is read from shared memory once per thread window and never again.
//   K <= 3 : the K accumulator planes rotate by unrolling the plane loop K times;
//   K >= 5 : they rotate by shifting once per plane (less code for the same arithmetic).
// Weights travel as kernel parameters and enter the FMAs as constant-bank operands.  For
// k = 3 the kernel is bound by instruction issue, not by HBM, so there the x taps of each
// output pair (x, x+1) run as one packed two-lane FMA (half the FMA instructions), and a
// thread holds 4 rows instead of 2 so the per-plane overhead spreads over 16 outputs.  A
// slot's first tap in a plane of its z-march (c = b = a = 0) is a plain product, so no
// accumulator is ever reset.
//
// Adjoint mode (ADJ): the same machinery evaluates dL/dx of the clamped correlation.  With
// the extension E (x_ext(j) = x(clamp(j)) on the domain padded by r), the forward filter is
// a plain correlation of x_ext, so its adjoint is E^T applied to the zero-padded correlation
// of gy with the flipped kernel, Z(j') = sum_d w[-d] gy0(j' + d) for j' in [-r, n+r)^3.
// E^T folds Z onto the volume: gx(j) = sum of Z(j') over the j' whose clamp is j.  The
// kernel computes Z on the volume itself, j' in [0, n)^3 (TMA zero-fills gy outside), where
// each Z(j') is the one contribution that lands on j' from inside, and stores it; the shell
// of positions outside the volume, j' in [-r, n+r)^3 \ [0, n)^3, is then folded slab by slab
// by k_adjoint_shell and added atomically to the face voxels it lands on.  (A kernel
// over the padded domain itself needed 3 x 5 column tiles instead of 2 x 4 at 128^3, and
// atomics wherever a position folds: twice the forward's time.)
//
// Compensated mode (COMP, integer destinations whose FP32 error bound could flip a code):
// every tap is added as an error-free product and sum (dot2_exact, the compensated dot
// product Dot2), each output keeps a (sum, error) pair, and the store takes the rounding
// decision on the pair in double-float arithmetic (comp_code).  A slot's first tap in a
// plane of its z-march sets the pair to the product and its rounding error (dot2_first_exact),
// which is what the addition to (0, 0) gives, so no slot is reset.  One output row per thread
// keeps the 2 x k x RX accumulators in registers.
#pragma once

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "vkt_internal.h"
#include "vkt_tile.cuh"

namespace vkt {
namespace dir {

constexpr int NT = 256;          // threads per CTA, 16 x 16
constexpr int BX = 16, BY = 16;
constexpr int STAGES = 4;        // raw tiles in flight per CTA

template <int K>
struct DenseW {
    float w[K * K * K];
};

struct DirectArgs {
    const void* src;
    void* dst;
    int nx, ny, nz;
    int ox0, oy0, oz0;     // origin of the output domain (0, or the padded domain's corner)
    int ex, ey, ez;        // extent of the output domain
    int sx0, sx1, sy1;     // forward: voxels with x in [sx0, sx1) and y < sy1 are stored
    int sfmt, dfmt;
    int zchunk;
    int gzv;               // z chunks per volume: blockIdx.z = volume * gzv + chunk
    int64_t vs_src, vs_dst;   // voxels from one volume of the batch to the next
    int use_tma;
    int rows;              // no tensor map: stages filled by per-row bulk copies (forward only)
    int withhold_first;    // fault injection: the first plane's TMA load is never issued
    float a0, a1, qmax;
    float a0lo, a1lo;      // compensated mode: low halves of a0, a1 (double-float pairs)
    unsigned* status;
};

// SHAPE 1: one output row per thread (64 x 16 tiles) for the plain k <= 3 kernels of
// volumes too small to give every SM a CTA (64^3: 4 tiles per plane instead of 1)
template <int K, bool COMP = false, int SHAPE = 0>
struct DirectCfg {
    static constexpr int RX = (K == 9 || (COMP && K >= 7)) ? 2 : 4;
    static constexpr int RY = (COMP || SHAPE == 1) ? 1 : ((K <= 3) ? 4 : 2);
    static constexpr bool ROT = K >= 5;
    // PAIR: the x taps run as packed two-lane FMAs over neighbouring outputs (x, x+1),
    // which halves the FMA instructions of a kernel whose time is instruction issue
    static constexpr bool PAIR = K == 3 && !COMP;
    static constexpr int TX = BX * RX, TY = BY * RY;
    using Geo = Brick<K, TX, TY>;
};

template <int K, bool COMP = false, int SHAPE = 0>
__host__ __device__ constexpr size_t direct_smem_bytes(int sfmt, bool rows)
{
    using Geo = typename DirectCfg<K, COMP, SHAPE>::Geo;
    return 128 + static_cast<size_t>(STAGES) * Geo::stage_bytes(sfmt, rows) +
           2 * static_cast<size_t>(Geo::FH) * Geo::FP * sizeof(float);
}

// SF/DF: source and destination formats fixed at compile time (-1: read from the arguments);
// LM: how stages are filled, fixed at compile time where known (the plane loop is unrolled,
// so code for unused ways of loading costs instruction cache): 0 = from the arguments
// (tensor map, row copies or plain loads), 1 = tensor map, 2 = row copies
constexpr int LM_ANY = 0, LM_TMA = 1, LM_ROWS = 2;
// ROI: the forward stores are bounded by the arguments' region fields; otherwise by the
// volume (known at compile time to start at column 0).  COMP: compensated accumulation
// into an integer destination (forward only).
template <int K, bool ADJ, int SF = -1, int DF = -1, int LM = LM_ANY, bool ROI = false,
          bool COMP = false, int SHAPE = 0>
__global__ void __launch_bounds__(NT)
    k_direct(const __grid_constant__ CUtensorMap tmap, const DirectArgs p, const DenseW<K> W)
{
    static_assert(!(COMP && ADJ), "the adjoint writes float32");
    using Cfg = DirectCfg<K, COMP, SHAPE>;
    using Geo = typename Cfg::Geo;
    constexpr int R = Geo::R, RX = Cfg::RX, RY = Cfg::RY;
    constexpr int FH = Geo::FH, FP = Geo::FP;

    extern __shared__ __align__(128) unsigned char smem[];
    const int sfmt = SF >= 0 ? SF : p.sfmt;
    const int dfmt = DF >= 0 ? DF : p.dfmt;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    const bool tma = LM == LM_TMA || (LM == LM_ANY && p.use_tma);
    const bool rows = !ADJ && (LM == LM_ROWS || (LM == LM_ANY && p.rows));
    const int rawb = Geo::stage_bytes(sfmt, rows);
    const uint32_t txb = Geo::raw_tx(sfmt);
    unsigned char* raw = smem + 128;
    float* F = reinterpret_cast<float*>(raw + STAGES * rawb);
    // a launch whose shared memory was sized for another tile shape records the mismatch
    // and does nothing (instead of running past the end of its shared memory)
    if (dynamic_smem_bytes() < direct_smem_bytes<K, COMP, SHAPE>(sfmt, rows)) {
        grid_dependency_wait();
        if (threadIdx.x == 0) atomicOr(p.status, STATUS_CONFIG);
        return;
    }

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int x0 = p.ox0 + blockIdx.x * Cfg::TX, y0 = p.oy0 + blockIdx.y * Cfg::TY;
    // volume of the batch and z chunk of this CTA; the volume's own source and destination
    const int vol = static_cast<int>(blockIdx.z) / p.gzv;
    const int zc0 = p.oz0 + (static_cast<int>(blockIdx.z) - vol * p.gzv) * p.zchunk;
    const void* src = static_cast<const unsigned char*>(p.src) + vol * p.vs_src * fmt_bytes(sfmt);
    void* dst = static_cast<unsigned char*>(p.dst) + vol * p.vs_dst * (ADJ ? 4 : fmt_bytes(dfmt));
    const int zc1 = min(zc0 + p.zchunk, p.oz0 + p.ez);
    if (zc0 >= zc1) return;
    const int pfirst = zc0 - R;
    const int nplanes = zc1 - zc0 + 2 * R;
    const int xa = fmt_xalign(sfmt);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        if (LM != LM_ROWS && p.use_tma) prefetch_tensor_map(&tmap);
    }
    __syncthreads();
    // set-up done: wait for the previous kernel on the stream (programmatic launch), let
    // the next one start its set-up
    grid_dependency_wait();
    launch_dependents();
    int issued = 0;   // planes handed to the TMA unit so far (thread 0 only)
    const uint64_t vol_bytes = static_cast<uint64_t>(p.nx) * p.ny * p.nz * fmt_bytes(sfmt);
    if (tma && tid == 0) {
        for (int s = 0; s < STAGES && s < nplanes; ++s, ++issued) {
            if (s == 0 && p.withhold_first) continue;
            mbar_arrive_expect_tx(&bars[s], txb);
            tma_load_4d(raw + s * rawb, &tmap, &bars[s], x0 - xa, y0 - R,
                        ADJ ? pfirst + s : clampi(pfirst + s, 0, p.nz - 1), vol);
        }
    } else if (rows) {
        for (int s = 0; s < STAGES && s < nplanes; ++s)
            issue_rows<Geo, NT>(raw + s * rawb, &bars[s], src, vol_bytes, sfmt, p.nx, p.ny,
                                p.nz, x0, y0, pfirst + s, tid);
        __syncthreads();   // every thread's expect_tx precedes the single arrival
        if (tid == 0)
            for (int s = 0; s < STAGES && s < nplanes; ++s, ++issued) mbar_arrive(&bars[s]);
    }
    // row copies issued in one plane get their arrival after the next plane's CTA barrier
    int pend = -1;

    ConvPlan<Geo, NT, !ADJ> plan;
    plan.init(sfmt, p.nx, p.ny, x0, y0, tid, rows);

    // Accumulators start at zero once; afterwards the first tap a plane's slot receives
    // (c = 0, b = 0, a = 0) is a plain product, which restarts the slot without a reset.
    // outputs (x, x+1) of a row share one float2, the operand of the packed FMAs
    static_assert(RX % 2 == 0, "outputs are paired along x");
    float2 acc[K][RY][RX / 2];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int i = 0; i < RY; ++i)
#pragma unroll
            for (int x = 0; x < RX / 2; ++x) acc[s][i][x] = make_float2(0.f, 0.f);
    auto lane = [&](int s, int i, int x) -> float& {
        return (x & 1) ? acc[s][i][x >> 1].y : acc[s][i][x >> 1].x;
    };
    // compensated mode: a (sum, error) pair per output, reset after its plane is stored
    float cs[COMP ? K : 1][RY][RX], cc[COMP ? K : 1][RY][RX];
    if constexpr (COMP) {
#pragma unroll
        for (int s = 0; s < K; ++s)
#pragma unroll
            for (int i = 0; i < RY; ++i)
#pragma unroll
                for (int x = 0; x < RX; ++x) cs[s][i][x] = cc[s][i][x] = 0.f;
    }

    const int ox = x0 + tx * RX;
    const int nvalid = (ROI ? p.sx1 : p.nx) - ox;
    const int first = (ROI && p.sx0 > ox) ? p.sx0 - ox : 0;   // leading columns outside the region
    const int yend = ROI ? p.sy1 : p.ny;
    bool failed = false;

    // One input plane: fetch, convert, multiply into the K output planes, retire one.
    auto plane = [&](const int it, const int u) {
        const int s = it % STAGES;
        const unsigned char* rs = raw + s * rawb;
        float* Fb = F + (it & 1) * FH * FP;
        bool ok = true;
        if (tma || rows) {
            ok = mbar_wait(&bars[s], (it / STAGES) & 1);
        } else {
            fill_raw_plain<Geo, NT, !ADJ>(const_cast<unsigned char*>(rs), src, sfmt, p.nx,
                                          p.ny, p.nz, x0, y0, pfirst + it, tid);
            __syncthreads();
        }
        if (ok) {
            if constexpr (!ADJ) {
                if (rows) {
                    const uint32_t zterm =
                        static_cast<uint32_t>(clampi(pfirst + it, 0, p.nz - 1)) *
                        static_cast<uint32_t>(p.ny) * static_cast<uint32_t>(p.nx);
                    plan.convert_rows(rs, sfmt, Fb, tid, p.nx, p.ny, x0, y0, zterm);
                } else {
                    plan.convert(rs, sfmt, Fb, tid);
                }
            } else {
                plan.convert(rs, sfmt, Fb, tid);
            }
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            return;
        }
        if (rows && tid == 0 && pend >= 0) {
            mbar_arrive(&bars[pend]);
            ++issued;
        }
        pend = -1;
        if (tma && tid == 0 && it + STAGES < nplanes) {
            mbar_arrive_expect_tx(&bars[s], txb);
            tma_load_4d(raw + s * rawb, &tmap, &bars[s], x0 - xa, y0 - R,
                        ADJ ? pfirst + it + STAGES : clampi(pfirst + it + STAGES, 0, p.nz - 1), vol);
            ++issued;
        } else if (rows && it + STAGES < nplanes) {
            issue_rows<Geo, NT>(raw + s * rawb, &bars[s], src, vol_bytes, sfmt, p.nx, p.ny,
                                p.nz, x0, y0, pfirst + it + STAGES, tid);
            pend = s;
        }
        // multiply the plane into the accumulators
        if constexpr (Cfg::PAIR && !COMP) {
            // row offset b outermost: the K*K weight pairs (w, w) of one b serve every output
            // row, so each pair is formed once per plane instead of once per input row (the
            // window rows are loaded K times instead of once; measured 1.4 % faster at k = 3)
#pragma unroll
            for (int b = 0; b < K; ++b) {
#pragma unroll
                for (int i = 0; i < RY; ++i) {
                    float win[RX + K - 1];
                    load_row<RX + K - 1, RX>(Fb + (ty * RY + i + b) * FP + tx * RX, win);
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const int sl = Cfg::ROT ? (K - 1 - c) : (((u - c + R) % K + K) % K);
#pragma unroll
                        for (int x = 0; x < RX; x += 2)
#pragma unroll
                            for (int a = 0; a < K; ++a) {
                                const float wv = W.w[(c * K + b) * K + a];
                                const float2 w2 = make_float2(wv, wv);
                                const float2 v2 = make_float2(win[x + a], win[x + a + 1]);
                                float2& d = acc[sl][i][x >> 1];
                                d = (c == 0 && b == 0 && a == 0) ? __fmul2_rn(w2, v2)
                                                                 : __ffma2_rn(w2, v2, d);
                            }
                    }
                }
            }
        } else {
#pragma unroll
        for (int j = 0; j < RY + K - 1; ++j) {
            float win[RX + K - 1];
            load_row<RX + K - 1, RX>(Fb + (ty * RY + j) * FP + tx * RX, win);
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const int b = j - i;
                if (b < 0 || b >= K) continue;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const int sl = Cfg::ROT ? (K - 1 - c) : (((u - c + R) % K + K) % K);
                    if constexpr (COMP) {
#pragma unroll
                        for (int x = 0; x < RX; ++x)
#pragma unroll
                            for (int a = 0; a < K; ++a) {
                                // a slot's first tap in its z-march sets it (no reset needed)
                                if (c == 0 && b == 0 && a == 0)
                                    dot2_first_exact(W.w[(c * K + b) * K + a], win[x + a],
                                                     cs[sl][i][x], cc[sl][i][x]);
                                else
                                    dot2_exact(W.w[(c * K + b) * K + a], win[x + a], cs[sl][i][x],
                                               cc[sl][i][x]);
                            }
                    } else if constexpr (Cfg::PAIR) {
#pragma unroll
                        for (int x = 0; x < RX; x += 2)
#pragma unroll
                            for (int a = 0; a < K; ++a) {
                                const float wv = W.w[(c * K + b) * K + a];
                                const float2 w2 = make_float2(wv, wv);
                                const float2 v2 = make_float2(win[x + a], win[x + a + 1]);
                                float2& d = acc[sl][i][x >> 1];
                                d = (c == 0 && b == 0 && a == 0) ? __fmul2_rn(w2, v2)
                                                                 : __ffma2_rn(w2, v2, d);
                            }
                    } else {
#pragma unroll
                        for (int x = 0; x < RX; ++x)
#pragma unroll
                            for (int a = 0; a < K; ++a) {
                                const float wv = W.w[(c * K + b) * K + a];
                                float& d = lane(sl, i, x);
                                d = (c == 0 && b == 0 && a == 0) ? wv * win[x + a]
                                                                 : fmaf(wv, win[x + a], d);
                            }
                    }
                }
            }
        }
        }
        // output plane it - 2R + zc0 is complete
        const int sl0 = Cfg::ROT ? 0 : (((u - R) % K + K) % K);
        if constexpr (COMP) {
            if (it >= 2 * R) {
                const int oz = pfirst + it - R;
#pragma unroll
                for (int i = 0; i < RY; ++i) {
                    const int oy = y0 + ty * RY + i;
                    if (oy < yend && nvalid > 0) {
                        const int64_t idx = (static_cast<int64_t>(oz) * p.ny + oy) * p.nx + ox;
#pragma unroll
                        for (int x = 0; x < RX; ++x) {
                            if (x < first || x >= nvalid) continue;
                            const unsigned code = comp_code(cs[sl0][i][x], cc[sl0][i][x], p.a0,
                                                            p.a0lo, p.a1, p.a1lo, p.qmax);
                            if (dfmt == FMT_U16)
                                static_cast<uint16_t*>(dst)[idx + x] = static_cast<uint16_t>(code);
                            else
                                static_cast<unsigned char*>(dst)[idx + x] = static_cast<unsigned char>(code);
                        }
                    }
                }
            }
            if constexpr (Cfg::ROT) {
#pragma unroll
                for (int q = 0; q + 1 < K; ++q)
#pragma unroll
                    for (int i = 0; i < RY; ++i)
#pragma unroll
                        for (int x = 0; x < RX; ++x) {
                            cs[q][i][x] = cs[q + 1][i][x];
                            cc[q][i][x] = cc[q + 1][i][x];
                        }
            }
            return;
        }
        if (it >= 2 * R) {
            const int oz = pfirst + it - R;
#pragma unroll
            for (int i = 0; i < RY; ++i) {
                const int oy = y0 + ty * RY + i;
                float row[RX];
#pragma unroll
                for (int x = 0; x < RX; ++x) row[x] = lane(sl0, i, x);
                if (oy < yend && nvalid > 0) {
                    const int64_t idx = (static_cast<int64_t>(oz) * p.ny + oy) * p.nx + ox;
                    store_row<RX>(dst, dfmt, idx, nvalid, row, p.a0, p.a1, p.qmax, first);
                }
            }
        }
        if (Cfg::ROT) {
#pragma unroll
            for (int q = 0; q + 1 < K; ++q)
#pragma unroll
                for (int i = 0; i < RY; ++i)
#pragma unroll
                    for (int x = 0; x < RX / 2; ++x) acc[q][i][x] = acc[q + 1][i][x];
        }
    };

    if (Cfg::ROT) {
        for (int it = 0; it < nplanes && !failed; ++it) plane(it, 0);
    } else {
        for (int g = 0; g * K < nplanes && !failed; ++g) {
#pragma unroll
            for (int u = 0; u < K; ++u) {
                const int it = g * K + u;
                if (it >= nplanes || failed) break;
                plane(it, u);
            }
        }
    }

    if (failed) {
        if (tid == 0) {
            atomicOr(p.status, STATUS_TIMEOUT);
            // a refill whose copies are in flight still needs its arrival before the drain
            if (pend >= 0) {
                mbar_arrive(&bars[pend]);
                ++issued;
            }
            // drain loads still in flight (bounded) before the CTA's smem is released:
            // the newest load issued to each stage completes that stage's current phase
            for (int it = issued - 1; it >= 0 && it >= issued - STAGES; --it)
                if (it != 0 || !p.withhold_first) mbar_wait(&bars[it % STAGES], (it / STAGES) & 1);
        }
        __syncthreads();
    }
}

// The adjoint's shell: the positions j' of [-r, n+r)^3 outside [0, n)^3, each of whose
// Z(j') = sum_d w[-d] gy0(j' + d) (W holds the flipped weights, gy0 is zero outside the
// volume) is added to gx(clamp(j')).  The shell is taken as three pairs of slabs: z outside
// the volume (x', y' anywhere in the padded range), then z inside and y outside, then z and
// y inside and x outside.  A slab folds along its own axis in one sum: for the low z face,
// sum over z' in [-r, 0) of Z(x', y', z') = sum over planes zz in [0, r) and taps (b, a) of
// Fz[zz][b][a] gy0(x' + a - r, y' + b - r, zz), with Fz[zz] = sum over c in [zz + r + 1, 2r]
// of W[c] (the taps of W that reach plane zz from below the volume); for the high face the
// planes are n - r + t, t in [0, r), with Fz[t] = sum over c in [0, t] of W[c]; likewise
// along y and x.  Each folded slab is a thin 2-D correlation: out(p, q) = sum over t < r and
// (u, v) in [0, k)^2 of F[t][u][v] S[t][p + u][q + v], S the r layers of gy next to the face.
// A CTA takes a 16 x 16 tile of one slab's outputs, stages its S (with halo, zero outside
// the volume) in shared memory, and adds each output atomically onto the face voxel it folds
// onto; blockIdx.x enumerates the tiles of the six slabs, blockIdx.y the volume of the batch.
// (One thread per shell position with k^3 taps read from global memory took 40 % of dL/dx at
// 8 x 128^3, k = 5: the x slabs' loads hit a different row in every lane.)
constexpr int SHELL_T = 16;   // output tile edge of the shell kernel (256 threads)

// The folded weights of the shell [face: low, high][axis: z, y, x][t][u][v] (t the layer of
// the folded axis, (u, v) the other two taps in (c, b, a) order), summed in float32 on the
// host in tap order and passed as launch constants, so the kernel's FMAs take them as
// constant operands.
template <int K>
struct ShellW {
    static constexpr int R = (K - 1) / 2;
    static constexpr int RKK = R > 0 ? R * K * K : 1;
    float f[6][RKK];
};

template <int K>
ShellW<K> fold_shell_weights(const DenseW<K>& W)
{
    constexpr int R = (K - 1) / 2, KK = K * K;
    ShellW<K> F;
    for (int face = 0; face < 2; ++face)
        for (int axis = 0; axis < 3; ++axis)
            for (int q = 0; q < R * KK; ++q) {
                const int t = q / KK, u = (q / K) % K, v = q % K;
                const int f0 = face == 0 ? t + R + 1 : 0, f1 = face == 0 ? 2 * R : t;
                float sum = 0.f;
                for (int f = f0; f <= f1; ++f) {
                    const int c = axis == 0 ? f : u;
                    const int b = axis == 0 ? u : (axis == 1 ? f : v);
                    const int a = axis == 2 ? f : v;
                    sum += W.w[(c * K + b) * K + a];
                }
                F.f[face * 3 + axis][q] = sum;
            }
    return F;
}

template <int K>
__host__ __device__ constexpr int shell_tiles(int nx, int ny, int nz, int* na, int* nb)
{
    constexpr int R = (K - 1) / 2, T = SHELL_T;
    const int px = nx + 2 * R, py = ny + 2 * R;
    const int a = 2 * ((py + T - 1) / T) * ((px + T - 1) / T);
    const int b2 = 2 * ((nz + T - 1) / T) * ((px + T - 1) / T);
    const int c = 2 * ((nz + T - 1) / T) * ((ny + T - 1) / T);
    if (na) *na = a;
    if (nb) *nb = b2;
    return a + b2 + c;
}

template <int K>
__global__ void __launch_bounds__(SHELL_T * SHELL_T)
    k_adjoint_shell(const float* __restrict__ gy, float* gx, int nx, int ny, int nz,
                    int64_t vs_src, int64_t vs_dst, const ShellW<K> FW)
{
    constexpr int R = (K - 1) / 2, T = SHELL_T, SP = T + 2 * R;
    __shared__ float S[R][SP][SP];
    const int tid = threadIdx.x;
    // programmatic launch: the main adjoint launch's stores are complete and visible
    grid_dependency_wait();
    launch_dependents();
    // this CTA's slab (0: z, 1: y, 2: x), face and tile
    int na = 0, nb = 0;
    shell_tiles<K>(nx, ny, nz, &na, &nb);
    const int px = nx + 2 * R, py = ny + 2 * R;
    int blk = blockIdx.x, slab, P, Q, offP, offQ;
    if (blk < na) {
        slab = 0; P = py; Q = px; offP = 2 * R; offQ = 2 * R;
    } else if (blk < na + nb) {
        blk -= na; slab = 1; P = nz; Q = px; offP = R; offQ = 2 * R;
    } else {
        blk -= na + nb; slab = 2; P = nz; Q = ny; offP = R; offQ = R;
    }
    const int tq = (Q + T - 1) / T, tp = (P + T - 1) / T;
    const int face = blk / (tp * tq);
    const int p0 = (blk / tq) % tp * T, q0 = blk % tq * T;
    const float* g = gy + static_cast<int64_t>(blockIdx.y) * vs_src;
    float* out = gx + static_cast<int64_t>(blockIdx.y) * vs_dst;
    // stage S[t][pp][qq] = gy0 at layer t of the face, p-axis p0 + pp - offP, q-axis
    // q0 + qq - offQ (x slabs: the layer index fastest, the r voxels of a row are adjacent)
    for (int e = tid; e < R * SP * SP; e += T * T) {
        int t, pp, qq;
        if (slab == 2) {
            t = e % R;
            qq = (e / R) % SP;
            pp = e / (R * SP);
        } else {
            qq = e % SP;
            pp = (e / SP) % SP;
            t = e / (SP * SP);
        }
        const int pi = p0 + pp - offP, qi = q0 + qq - offQ;
        int x, y, z;
        if (slab == 0) {
            x = qi; y = pi; z = face == 0 ? t : nz - R + t;
        } else if (slab == 1) {
            x = qi; y = face == 0 ? t : ny - R + t; z = pi;
        } else {
            x = face == 0 ? t : nx - R + t; y = qi; z = pi;
        }
        S[t][pp][qq] = (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz)
                           ? __ldg(g + (static_cast<int64_t>(z) * ny + y) * nx + x)
                           : 0.f;
    }
    __syncthreads();
    const int tx = tid % T, ty = tid / T;
    const int p = p0 + ty, q = q0 + tx;
    if (p >= P || q >= Q) return;
    // the (face, slab) weights as compile-time indices of the launch constants
    float acc = 0.f;
    auto fold = [&](auto fs) {
        constexpr int FS = decltype(fs)::value;
#pragma unroll
        for (int t = 0; t < R; ++t)
#pragma unroll
            for (int u = 0; u < K; ++u)
#pragma unroll
                for (int v = 0; v < K; ++v)
                    acc = fmaf(FW.f[FS][(t * K + u) * K + v], S[t][ty + u][tx + v], acc);
    };
    switch (face * 3 + slab) {
    case 0: fold(std::integral_constant<int, 0>{}); break;
    case 1: fold(std::integral_constant<int, 1>{}); break;
    case 2: fold(std::integral_constant<int, 2>{}); break;
    case 3: fold(std::integral_constant<int, 3>{}); break;
    case 4: fold(std::integral_constant<int, 4>{}); break;
    default: fold(std::integral_constant<int, 5>{}); break;
    }
    int ox, oy, oz;
    if (slab == 0) {
        ox = clampi(q - R, 0, nx - 1); oy = clampi(p - R, 0, ny - 1); oz = face == 0 ? 0 : nz - 1;
    } else if (slab == 1) {
        ox = clampi(q - R, 0, nx - 1); oy = face == 0 ? 0 : ny - 1; oz = p;
    } else {
        ox = face == 0 ? 0 : nx - 1; oy = q; oz = p;
    }
    atomicAdd(out + (static_cast<int64_t>(oz) * ny + oy) * nx + ox, acc);
}

// True if the job's default k <= 3 tiles (64 x 64), in chunks of at least 8 planes, give
// fewer CTAs than the GPU has SMs: the one-row-per-thread shape then runs 4x as many CTAs.
inline bool direct_small(const Job& job, int sms)
{
    int rx0, ry0, rz0, rx1, ry1, rz1;
    job_region(job, rx0, ry0, rz0, rx1, ry1, rz1);
    const long tiles = static_cast<long>((rx1 - rx0 + 63) / 64) * ((ry1 - ry0 + 63) / 64) *
                       std::max(job.nvol, 1);
    const long cap8 = std::max((rz1 - rz0) / 8, 1);
    return tiles * cap8 < sms;
}

// One launch of the direct kernel over the job's region (forward) or over the padded
// domain (adjoint); COMP: compensated accumulation into an integer destination.
template <int K, bool ADJ, bool COMP = false, int SHAPE = 0>
vktError launch_k(const Job& job, const float* w, const Ctx& ctx)
{
    static_assert(!(COMP && ADJ), "the adjoint writes float32");
    using Cfg = DirectCfg<K, COMP, SHAPE>;
    using Geo = typename Cfg::Geo;
    constexpr int R = Geo::R;
    DirectArgs a;
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
    a.a0lo = job.a0lo;
    a.a1lo = job.a1lo;
    a.status = ctx.status;
    a.withhold_first = (ctx.debug & VKT_DEBUG_INJECT_WAIT_TIMEOUT) ? 1 : 0;
    if (ADJ) {
        // Z on the volume's own positions (the shell outside it: k_adjoint_shell)
        a.ox0 = a.oy0 = a.oz0 = 0;
        a.ex = job.nx;
        a.ey = job.ny;
        a.ez = job.nz;
        a.sx0 = 0;
        a.sx1 = job.nx;
        a.sy1 = job.ny;
    } else {
        // output region; the tiles start on a 16-byte boundary left of it (tensor-map boxes
        // start there) and store only inside it
        int rx0, ry0, rz0, rx1, ry1, rz1;
        job_region(job, rx0, ry0, rz0, rx1, ry1, rz1);
        a.ox0 = rx0 - rx0 % fmt_xalign(job.sfmt);
        a.oy0 = ry0;
        a.oz0 = rz0;
        a.ex = rx1 - a.ox0;
        a.ey = ry1 - ry0;
        a.ez = rz1 - rz0;
        a.sx0 = rx0;
        a.sx1 = rx1;
        a.sy1 = ry1;
    }
    DenseW<K> W;
    const int kk = K * K * K;
    for (int i = 0; i < kk; ++i) W.w[i] = ADJ ? w[kk - 1 - i] : w[i];   // adjoint: w[-d]

    const int gx = (a.ex + Cfg::TX - 1) / Cfg::TX;
    const int gy = (a.ey + Cfg::TY - 1) / Cfg::TY;
    const int sms = ctx.sms;
    const int nvol = std::max(job.nvol, 1);
    a.vs_src = job.vs_src;
    a.vs_dst = job.vs_dst;

    alignas(64) CUtensorMap map;
    const int rawx = Geo::raw_w(job.sfmt);
    const int es = fmt_bytes(job.sfmt);
    auto encode = [&](const void* base, int nv) {
        return encode_tensor_map(&map, job.sfmt, base, job.nx, job.ny, job.nz, nv, job.vs_src, rawx,
                                 Geo::FH, 1);
    };
    // the tensor map spans the volumes of one launch, at most 65535 / gz (the grid's z extent);
    // encoded for the whole batch first and re-encoded per launch once gz is known
    a.use_tma = encode(job.src, std::min(nvol, 65535)) ? 1 : 0;
    if (!a.use_tma) memset(&map, 0, sizeof(map));
    // rows that no tensor map can describe are still fetched asynchronously, one bulk copy
    // per row, when every volume starts on a 16-byte boundary (forward only: the adjoint
    // needs the zero extension a tensor map or the plain loads give)
    a.rows = (!ADJ && !a.use_tma && reinterpret_cast<uintptr_t>(job.src) % 16 == 0 &&
              (job.vs_src * es) % 16 == 0)
                 ? 1
                 : 0;

    const size_t smem = direct_smem_bytes<K, COMP, SHAPE>(job.sfmt, a.rows != 0);
    // the common float32 destinations get kernels with their formats compiled in
    // tensor-map jobs get kernels without the other ways of loading, and so do row-copy
    // jobs of the compiled-in formats; plain-load jobs take the run-time variant
    auto kern = a.use_tma ? k_direct<K, ADJ, -1, -1, LM_TMA, false, COMP, SHAPE>
                          : k_direct<K, ADJ, -1, -1, LM_ANY, false, COMP, SHAPE>;
    if constexpr (!ADJ) {
        if (job.roi) kern = k_direct<K, ADJ, -1, -1, LM_ANY, true, COMP, SHAPE>;   // reads the region fields
    }
    if constexpr (!ADJ && !COMP && K >= 3 && K <= 5) {
        // region tensor-map jobs of the common float32 destinations: formats compiled in
        if (job.roi && a.use_tma && job.dfmt == FMT_F32 && job.sfmt == FMT_U8)
            kern = k_direct<K, ADJ, FMT_U8, FMT_F32, LM_TMA, true, false, SHAPE>;
        if (job.roi && a.use_tma && job.dfmt == FMT_F32 && job.sfmt == FMT_F32)
            kern = k_direct<K, ADJ, FMT_F32, FMT_F32, LM_TMA, true, false, SHAPE>;
    }
    if constexpr (ADJ && K >= 3 && K <= 5) {
        // the adjoint reads and writes float32: formats compiled in for tensor-map jobs
        if (a.use_tma) kern = k_direct<K, ADJ, FMT_F32, FMT_F32, LM_TMA, false, false, SHAPE>;
    }
    if constexpr (!ADJ && !COMP && K >= 3 && K <= 5) {
        if (!job.roi && job.dfmt == FMT_F32 && job.sfmt == FMT_U8) {
            if (a.use_tma) kern = k_direct<K, ADJ, FMT_U8, FMT_F32, LM_TMA, false, false, SHAPE>;
            else if (a.rows) kern = k_direct<K, ADJ, FMT_U8, FMT_F32, LM_ROWS, false, false, SHAPE>;
        }
        if (!job.roi && job.dfmt == FMT_F32 && job.sfmt == FMT_F32) {
            if (a.use_tma) kern = k_direct<K, ADJ, FMT_F32, FMT_F32, LM_TMA, false, false, SHAPE>;
            else if (a.rows) kern = k_direct<K, ADJ, FMT_F32, FMT_F32, LM_ROWS, false, false, SHAPE>;
        }
    }
    int per_sm = 1;
    const vktError ve = prepare_kernel(ctx, reinterpret_cast<const void*>(kern), NT, smem, &per_sm);
    if (ve != VKT_NO_ERROR) return ve;
    cudaError_t e = cudaSuccess;
    a.zchunk = job.zchunk > 0 ? std::min(job.zchunk, a.ez)
                              : zchunk_direct(static_cast<long>(gx) * gy * nvol, a.ez, sms, per_sm, R);
    const int gz = (a.ez + a.zchunk - 1) / a.zchunk;
    a.gzv = gz;
    const int per_launch = std::max(1, 65535 / gz);
    if (a.use_tma && per_launch < nvol && !encode(job.src, per_launch)) return VKT_ERROR_CUDA;
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] direct%s k=%d grid=(%d,%d,%d) zchunk=%d smem=%zu tma=%d rows=%d withhold=%d\n",
                ADJ ? "-adjoint" : (COMP ? "-compensated" : ""), K, gx, gy, gz, a.zchunk, smem,
                a.use_tma, a.rows, a.withhold_first);
    const DirectArgs a0 = a;
    for (int v0 = 0; v0 < nvol; v0 += per_launch) {
        const int nv = std::min(per_launch, nvol - v0);
        a.src = static_cast<const unsigned char*>(a0.src) + v0 * a0.vs_src * es;
        a.dst = static_cast<unsigned char*>(a0.dst) + v0 * a0.vs_dst * (ADJ ? 4 : fmt_bytes(job.dfmt));
        if (v0 > 0 && a.use_tma && !encode(a.src, nv)) return VKT_ERROR_CUDA;
        e = launch_pdl(kern, dim3(gx, gy, gz * nv), dim3(NT), smem, ctx.stream, map, a, W);
        count_launches(1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return from_cuda(e);
        if constexpr (ADJ && R > 0) {
            // the shell outside the volumes, folded onto their faces after the main launch
            const int tiles = shell_tiles<K>(job.nx, job.ny, job.nz, nullptr, nullptr);
            e = launch_pdl(k_adjoint_shell<K>, dim3(tiles, nv), dim3(SHELL_T * SHELL_T), 0, ctx.stream,
                           static_cast<const float*>(a.src), static_cast<float*>(a.dst), job.nx,
                           job.ny, job.nz, a0.vs_src, a0.vs_dst, fold_shell_weights<K>(W));
            count_launches(1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) return from_cuda(e);
        }
    }
    return VKT_NO_ERROR;
}

}  // namespace dir
}  // namespace vkt
