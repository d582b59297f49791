// vkt_tc.cu -- ApplyFilter on the tcgen05 tensor cores for dense k^3 filters (k = 5, 7, 9)
// on float32 volumes, with a split FP16 hi/lo operand scheme that keeps the result within
// the FP32 path's accuracy.
//
// Formulation.  Fix one input plane z' and one kernel row offset b (dy = b - r).  For the
// 8 outputs x_o of an x tile, the x taps of every kernel plane c are a banded Toeplitz
// product over a 16-wide input window:
//     D[m, (c, j)] += sum_kk  A_b[m, kk] * T_b[kk, (c, j)]
//     A_b[m, kk]   = v(x0 - 4 + 8t + kk, y0 + m + dy, z')          (input rows shifted by dy)
//     T_b[kk,(c,j)] = w[c][b][kk - j - 4 + r]   (zero outside the band)
// so one 128 x N x 16 MMA (M = 128 output rows, N = 8 * slots, slots >= k) yields the
// contribution of plane z' to the k output planes z' - c + r at once.  Summing over b and
// over the three split products A_hi T_hi + A_hi T_lo + A_lo T_hi (each operand split as
// hi = fp16(x s), lo = fp16(x s - hi), s a power of two) happens in the TMEM accumulator;
// the epilogue scales back and adds the k slot columns into k rotating register
// accumulators, one of which completes per input plane (z-march).
//
// Warp roles (448 threads, one CTA per SM, persistent over (x, y, z-chunk) work items):
//   warp 0       TMEM allocation; lane 0 issues TMA loads of f32 plane tiles
//   warp 1       lane 0 issues the MMAs and commits
//   warps 2..5   convert a plane tile to fp16 hi/lo operands (clamp-to-edge, scale)
//   warps 6..13  epilogue: TMEM -> registers, z-march accumulate, store
// Every wait is bounded; on a timeout the CTA records it, drains what it issued and exits.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "vkt_internal.h"
#include "vkt_tile.cuh"

namespace vkt {
namespace {

constexpr int MROWS = 128;                 // output rows per tile (MMA M)
constexpr int XT = 2;                      // x tiles of 8 outputs per work item
constexpr int NCH = XT + 1;                // 8-wide input chunks per plane tile
constexpr int STAGES = 4;
constexpr int NTHREADS = 448;
constexpr int CONV_WARP0 = 2, NCONV = 128;
constexpr int EPI_WARP0 = 6, NEPI = 256;
constexpr int SC_RING = 8;

template <int K>
struct TcCfg {
    static constexpr int R = (K - 1) / 2;
    static constexpr int ROWS = MROWS + 2 * R;            // input rows of a plane tile
    static constexpr int SLOTS = ((K + 1) / 2) * 2;       // even, so N is a multiple of 16
    static constexpr int N = SLOTS * 8;
    // CAT: the hi*hi and hi*lo products share one MMA of width 2N over the stacked
    // operand [T_hi | T_lo], so A_hi is read once per (dy, x tile); the D columns [0,N)
    // then hold hi*hi + lo*hi and [N,2N) hold hi*lo.  Measured slower on GB300 (the
    // epilogue reads twice the columns), so it is off.
    static constexpr bool CAT = false;
    static constexpr int DN = CAT ? 2 * N : N;          // TMEM columns per (buffer, x tile)
    static constexpr int DBUF = 3;                       // TMEM accumulator buffers
    static_assert(DBUF * XT * DN <= 512, "TMEM holds 512 columns");
    static constexpr int TMEM_COLS = (DBUF * XT * DN <= 256) ? 256 : 512;
    static constexpr int STAGE_BYTES = ((ROWS * NCH * 8 * 4) + 1023) & ~1023;
    static constexpr int STAGE_TX = ROWS * NCH * 8 * 4;
    static constexpr int OP_BYTES = ((NCH * ROWS * 16) + 1023) & ~1023;   // one fp16 plane
    static constexpr int B_BYTES = 2 * N * 16;                            // one Toeplitz (hi or lo)
    // converter items: (chunk, row, half) with the half fastest, 4 values each, so that a
    // quarter warp's 16-byte reads of the stage (rows 96 bytes apart) and its 8-byte writes
    // of the operand planes touch distinct banks
    static constexpr int UNITS = NCH * ROWS * 2;
    static constexpr int UPT = (UNITS + NCONV - 1) / NCONV;               // items per thread
    // shared memory map
    static constexpr int OFF_STAGE = 1024;
    static constexpr int OFF_OP = OFF_STAGE + STAGES * STAGE_BYTES;       // [2 bufs][hi,lo]
    static constexpr int OFF_B = OFF_OP + 4 * OP_BYTES;                   // [K][hi,lo]
    static constexpr int SMEM = OFF_B + ((2 * K * B_BYTES + 1023) & ~1023);
};

template <int K>
struct TcW {
    float w[K * K * K];
};

struct TcArgs {
    float* dst;
    int nx, ny, nz;
    int items_x, items_y, items_z, nitems, zchunk;
    int wexp;            // weights are scaled by 2^wexp before splitting
    unsigned* status;
};

// header of the shared memory map (first 1024 bytes)
struct TcHeader {
    uint64_t stage_full[STAGES];
    uint64_t stage_empty[STAGES];
    uint64_t op_full[2];
    uint64_t op_empty[2];
    uint64_t d_full[3];
    uint64_t d_free[3];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
    int conv_ok;
    int sc[SC_RING];     // per-plane scale exponents written by the converters
    int dsc[3];          // scale exponent of the plane in each TMEM buffer
    float red[2][4];     // converter max reduction
};
static_assert(sizeof(TcHeader) <= 1024, "header");

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // tcgen05 shared-memory matrix descriptor, no swizzle, K-major canonical layout of
    // 8-row x 16-byte core matrices: start, leading (K) byte offset, stride (M/N) byte
    // offset, all >> 4; bits 46-48 hold the fixed value 0b001.
    uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;
}

__device__ __forceinline__ void umma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 columns of this warp's 32 lanes into v[0..15]; complete after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float* v)
{
    uint32_t* r = reinterpret_cast<uint32_t*>(v);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void named_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Bounded wait that also gives up when another role has aborted.  The waiting thread asks
// to be suspended (up to the hint) instead of polling, so idle roles do not take issue
// slots from the MMA-issuing warp on their sub-partition.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                              unsigned* status)
{
    if (mbar_try_wait_sleep(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_sleep(bar, parity)) {
        if (*abort_flag) return false;
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            *abort_flag = 1;
            atomicOr(status, STATUS_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

template <int K>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc(const __grid_constant__ CUtensorMap tmap, const TcArgs p, const TcW<K> W)
{
    using C = TcCfg<K>;
    constexpr int R = C::R, ROWS = C::ROWS, N = C::N;
    extern __shared__ __align__(1024) unsigned char smem[];
    TcHeader& h = *reinterpret_cast<TcHeader*>(smem);
    volatile int* abort_flag = &h.abort_flag;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

    // ---- set-up: barriers, TMEM, Toeplitz operands
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&h.stage_full[s], 1);
            mbar_init(&h.stage_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&h.op_full[b], 1);
            mbar_init(&h.op_empty[b], 1);
        }
        for (int b = 0; b < C::DBUF; ++b) {
            mbar_init(&h.d_full[b], 2);          // MMA completion + the issuer's scale hand-off
            mbar_init(&h.d_free[b], NEPI / 32);
        }
        mbar_init(&h.drain, 1);
        h.abort_flag = 0;
        fence_mbar_init();
        prefetch_tensor_map(&tmap);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&h.tmem_base)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    {
        // T_b hi/lo, K-major [kc][n][8 halves] with n = (slot c, j) and entry kk = kc*8 + e.
        // CAT: one matrix per b with 2N rows per kc chunk (rows [0,N) hi, [N,2N) lo);
        // otherwise the hi matrix followed by the lo matrix.
        const float sw = pow2f(p.wexp);
        __half* B = reinterpret_cast<__half*>(smem + C::OFF_B);
        const int per_b = 2 * N * 8;
        for (int i = tid; i < K * per_b; i += NTHREADS) {
            const int b = i / per_b, rem = i - b * per_b;
            const int kc = rem / (N * 8), n = (rem / 8) % N, e = rem % 8;
            const int c = n / 8, j = n % 8, kk = kc * 8 + e;
            const int a = kk - j - 4 + R;
            float v = 0.f;
            if (c < K && a >= 0 && a < K) v = W.w[(c * K + b) * K + a] * sw;
            const __half hi = __float2half_rn(v);
            const __half lo = __float2half_rn(v - __half2float(hi));
            if (C::CAT) {
                __half* Bb = B + b * 2 * (C::B_BYTES / 2);
                Bb[(kc * 2 * N + n) * 8 + e] = hi;
                Bb[(kc * 2 * N + N + n) * 8 + e] = lo;
            } else {
                B[(2 * b + 0) * (C::B_BYTES / 2) + rem] = hi;
                B[(2 * b + 1) * (C::B_BYTES / 2) + rem] = lo;
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = h.tmem_base;
    const uint32_t sbase = smem_u32(smem);

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < p.nitems && ok; item += gridDim.x) {
                const int xi = item % p.items_x, yi = (item / p.items_x) % p.items_y;
                const int zi = item / (p.items_x * p.items_y);
                const int x0 = xi * 8 * XT, y0 = yi * MROWS, zc0 = zi * p.zchunk;
                const int zc1 = min(zc0 + p.zchunk, p.nz);
                const int nplanes = zc1 - zc0 + 2 * R;
                for (int it = 0; it < nplanes; ++it, ++g) {
                    const int s = g % STAGES;
                    if (g >= STAGES && !wait_or_abort(&h.stage_empty[s], ((g / STAGES) - 1) & 1,
                                                      abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&h.stage_full[s], C::STAGE_TX);
                    tma_load_3d(smem + C::OFF_STAGE + s * C::STAGE_BYTES, &tmap, &h.stage_full[s],
                                x0 - 4, y0 - R, clampi(zc0 - R + it, 0, p.nz - 1));
                }
            }
            // drain: every issued load completes its stage (bounded, no abort check)
            for (uint32_t q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
                mbar_wait(&h.stage_full[q % STAGES], (q / STAGES) & 1);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            // idesc: D f32, A f16, B f16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
            const uint32_t idesc = (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) |
                                   (static_cast<uint32_t>(MROWS >> 4) << 24);
            const uint32_t idesc2 = (1u << 4) | (static_cast<uint32_t>((2 * N) >> 3) << 17) |
                                    (static_cast<uint32_t>(MROWS >> 4) << 24);
            // Descriptors are built once: B per (dy, part) for the whole kernel, A as a per-
            // buffer base to which each MMA adds its compile-time offset in the 14-bit start
            // address field (addresses stay below 256 KB, so the add never carries out), so
            // the issuing thread spends about one instruction per MMA.
            uint64_t bdesc[2 * K];
#pragma unroll
            for (int b = 0; b < K; ++b) {
                const uint32_t bb = sbase + C::OFF_B + 2 * b * C::B_BYTES;
                if (C::CAT) {
                    bdesc[2 * b] = umma_desc(bb, 2 * N * 16, 128);
                    bdesc[2 * b + 1] = bdesc[2 * b];
                } else {
                    bdesc[2 * b] = umma_desc(bb, N * 16, 128);
                    bdesc[2 * b + 1] = umma_desc(bb + C::B_BYTES, N * 16, 128);
                }
            }
            uint64_t abase[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) abase[q] = umma_desc(sbase + C::OFF_OP + q * C::OP_BYTES, ROWS * 16, 128);
            uint32_t g = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < p.nitems && ok; item += gridDim.x) {
                const int zi = item / (p.items_x * p.items_y);
                const int zc0 = zi * p.zchunk, zc1 = min(zc0 + p.zchunk, p.nz);
                const int nplanes = zc1 - zc0 + 2 * R;
                for (int it = 0; it < nplanes; ++it, ++g) {
                    const int ob = g & 1, db = g % C::DBUF;
                    if (!wait_or_abort(&h.op_full[ob], (g >> 1) & 1, abort_flag, p.status) ||
                        (g >= C::DBUF && !wait_or_abort(&h.d_free[db], ((g / C::DBUF) - 1) & 1,
                                                        abort_flag, p.status))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ahi0 = ob ? abase[2] : abase[0];
                    const uint64_t alo0 = ob ? abase[3] : abase[1];
                    const uint32_t d0 = tbase + static_cast<uint32_t>(db * XT * C::DN);
#pragma unroll
                    for (int t = 0; t < XT; ++t) {
                        const uint32_t dt = d0 + static_cast<uint32_t>(t * C::DN);
#pragma unroll
                        for (int b = 0; b < K; ++b) {
                            const uint64_t aoff = static_cast<uint64_t>((t * (ROWS * 16) + b * 16) >> 4);
                            if (C::CAT) {
                                umma_f16(dt, ahi0 + aoff, bdesc[2 * b], idesc2, b > 0 ? 1u : 0u);
                                umma_f16(dt, alo0 + aoff, bdesc[2 * b], idesc, 1u);
                            } else {
                                umma_f16(dt, ahi0 + aoff, bdesc[2 * b], idesc, b > 0 ? 1u : 0u);
                                umma_f16(dt, ahi0 + aoff, bdesc[2 * b + 1], idesc, 1u);
                                umma_f16(dt, alo0 + aoff, bdesc[2 * b], idesc, 1u);
                            }
                        }
                    }
                    umma_commit(&h.op_empty[ob]);
                    h.dsc[db] = h.sc[g % SC_RING];
                    umma_commit(&h.d_full[db]);
                    mbar_arrive(&h.d_full[db]);
                }
            }
            // drain: all MMAs issued so far complete before TMEM is released
            umma_commit(&h.drain);
            mbar_wait(&h.drain, 0);
        }
    } else if (warp < EPI_WARP0) {
        // ---------------- converters: f32 tile -> fp16 hi/lo operand planes
        const int ct = tid - CONV_WARP0 * 32;           // 0..127
        const int cw = ct / 32;
        uint32_t g = 0;
        for (int item = blockIdx.x; item < p.nitems; item += gridDim.x) {
            const int xi = item % p.items_x, yi = (item / p.items_x) % p.items_y;
            const int zi = item / (p.items_x * p.items_y);
            const int x0 = xi * 8 * XT, y0 = yi * MROWS, zc0 = zi * p.zchunk;
            const int zc1 = min(zc0 + p.zchunk, p.nz);
            const int nplanes = zc1 - zc0 + 2 * R;
            bool ok = true;
            for (int it = 0; it < nplanes; ++it, ++g) {
                const int s = g % STAGES, ob = g & 1;
                if (ct == 0) {
                    bool w = wait_or_abort(&h.stage_full[s], (g / STAGES) & 1, abort_flag, p.status);
                    if (w && g >= 2)
                        w = wait_or_abort(&h.op_empty[ob], ((g >> 1) - 1) & 1, abort_flag, p.status);
                    h.conv_ok = w ? 1 : 0;
                }
                named_sync(1, NCONV);
                if (!*reinterpret_cast<volatile int*>(&h.conv_ok)) {
                    ok = false;
                    break;
                }
                const float* st = reinterpret_cast<const float*>(smem + C::OFF_STAGE + s * C::STAGE_BYTES);
                float v[C::UPT][4];
                float mx = 0.f;
#pragma unroll
                for (int q = 0; q < C::UPT; ++q) {
                    const int u = ct + q * NCONV;
                    if (u < C::UNITS) {
                        const int hf = u & 1, cr = u >> 1;
                        const int ch = cr / ROWS, row = cr - ch * ROWS;
                        const int gy = clampi(y0 - R + row, 0, p.ny - 1);
                        const float* sr = st + (gy - (y0 - R)) * (NCH * 8);
                        const int gx0 = x0 - 4 + 8 * ch + 4 * hf;
                        if (gx0 >= 0 && gx0 + 3 < p.nx) {
                            const float4 a = *reinterpret_cast<const float4*>(sr + 8 * ch + 4 * hf);
                            v[q][0] = a.x; v[q][1] = a.y; v[q][2] = a.z; v[q][3] = a.w;
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                v[q][e] = sr[clampi(gx0 + e, 0, p.nx - 1) - (x0 - 4)];
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fabsf(v[q][e]));
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if ((ct & 31) == 0) h.red[g & 1][cw] = mx;
                named_sync(1, NCONV);
                if (ct == 0) mbar_arrive(&h.stage_empty[s]);
                mx = fmaxf(fmaxf(h.red[g & 1][0], h.red[g & 1][1]), fmaxf(h.red[g & 1][2], h.red[g & 1][3]));
                // scale exponent: max|x| * 2^e in [2^13, 2^14)
                int ex = 0;
                int e = 0;
                if (mx > 0.f && mx <= 3.0e38f) {
                    frexpf(mx, &ex);
                    e = min(max(14 - ex, -100), 100);
                }
                if (ct == 0) h.sc[g % SC_RING] = e;
                const float sx = pow2f(e);
                unsigned char* ohi = smem + C::OFF_OP + (2 * ob + 0) * C::OP_BYTES;
                unsigned char* olo = smem + C::OFF_OP + (2 * ob + 1) * C::OP_BYTES;
#pragma unroll
                for (int q = 0; q < C::UPT; ++q) {
                    const int u = ct + q * NCONV;
                    if (u < C::UNITS) {
                        uint32_t hw[2], lw[2];
#pragma unroll
                        for (int e2 = 0; e2 < 2; ++e2) {
                            const float a = v[q][2 * e2] * sx, b = v[q][2 * e2 + 1] * sx;
                            const __half ah = __float2half_rn(a), bh = __float2half_rn(b);
                            const __half al = __float2half_rn(a - __half2float(ah));
                            const __half bl = __float2half_rn(b - __half2float(bh));
                            hw[e2] = static_cast<uint32_t>(__half_as_ushort(ah)) |
                                     (static_cast<uint32_t>(__half_as_ushort(bh)) << 16);
                            lw[e2] = static_cast<uint32_t>(__half_as_ushort(al)) |
                                     (static_cast<uint32_t>(__half_as_ushort(bl)) << 16);
                        }
                        // item u = (chunk, row, half) lands at chunk*ROWS*16 + row*16 + half*8 = u*8
                        *reinterpret_cast<uint2*>(ohi + u * 8) = make_uint2(hw[0], hw[1]);
                        *reinterpret_cast<uint2*>(olo + u * 8) = make_uint2(lw[0], lw[1]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                named_sync(1, NCONV);
                if (ct == 0) mbar_arrive(&h.op_full[ob]);
            }
            if (!ok) break;
        }
    } else {
        // ---------------- epilogue
        const int et = tid - EPI_WARP0 * 32;            // 0..255
        const int t = et / 128;                          // x tile
        const int quad = warp & 3;                       // TMEM lane quadrant of this warp
        const int m = quad * 32 + lane;                  // output row within the tile
        const uint32_t lane_addr = static_cast<uint32_t>(quad * 32) << 16;
        uint32_t g = 0;
        float acc[K][8];
        bool ok = true;
        for (int item = blockIdx.x; item < p.nitems && ok; item += gridDim.x) {
            const int xi = item % p.items_x, yi = (item / p.items_x) % p.items_y;
            const int zi = item / (p.items_x * p.items_y);
            const int x0 = xi * 8 * XT, y0 = yi * MROWS, zc0 = zi * p.zchunk;
            const int zc1 = min(zc0 + p.zchunk, p.nz);
            const int nplanes = zc1 - zc0 + 2 * R;
            const int oy = y0 + m, ox = x0 + 8 * t;
            const int nvalid = p.nx - ox;
#pragma unroll
            for (int c = 0; c < K; ++c)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[c][j] = 0.f;

            auto plane = [&](const int it, const int u) {
                const int db = g % C::DBUF;
                int w = 1;
                if (lane == 0) w = wait_or_abort(&h.d_full[db], (g / C::DBUF) & 1, abort_flag, p.status) ? 1 : 0;
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) {
                    ok = false;
                    return;
                }
                tc_fence_after();
                const float inv = pow2f(-(h.dsc[db] + p.wexp));
                const uint32_t col = tbase + lane_addr + static_cast<uint32_t>((db * XT + t) * C::DN);
                // two 16-column loads in flight per wait: slots 4q .. 4q+3
#pragma unroll
                for (int q = 0; q < (N / 16 + 1) / 2; ++q) {
                    float d[32];
                    const bool two = 2 * q + 1 < N / 16;
                    tmem_ld16_nowait(col + 32 * q, d);
                    if (two) tmem_ld16_nowait(col + 32 * q + 16, d + 16);
                    tmem_wait_ld();
#pragma unroll
                    for (int h2 = 0; h2 < 4; ++h2) {
                        const int c = 4 * q + h2;
                        if (c < K && (h2 < 2 || two)) {
                            const int sl = ((u - c + R) % K + K) % K;
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[sl][j] = fmaf(d[8 * h2 + j], inv, acc[sl][j]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&h.d_free[db]);
                const int sl0 = ((u - R) % K + K) % K;
                if (it >= 2 * R && oy < p.ny && nvalid > 0) {
                    const int oz = zc0 + it - 2 * R;
                    float* d = p.dst + (static_cast<int64_t>(oz) * p.ny + oy) * p.nx + ox;
                    if (nvalid >= 8 && ((reinterpret_cast<uintptr_t>(d) & 15) == 0)) {
                        reinterpret_cast<float4*>(d)[0] = make_float4(acc[sl0][0], acc[sl0][1], acc[sl0][2], acc[sl0][3]);
                        reinterpret_cast<float4*>(d)[1] = make_float4(acc[sl0][4], acc[sl0][5], acc[sl0][6], acc[sl0][7]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (j < nvalid) d[j] = acc[sl0][j];
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[sl0][j] = 0.f;
                ++g;
            };

            for (int g0 = 0; g0 < nplanes && ok; g0 += K) {
#pragma unroll
                for (int u = 0; u < K; ++u) {
                    if (g0 + u >= nplanes || !ok) break;
                    plane(g0 + u, u);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(C::TMEM_COLS)
                     : "memory");
    }
}

template <int K>
vktError launch_k(const Job& job, const float* w, const Ctx& ctx)
{
    using C = TcCfg<K>;
    TcArgs a;
    a.dst = static_cast<float*>(job.dst);
    a.nx = job.nx;
    a.ny = job.ny;
    a.nz = job.nz;
    a.status = ctx.status;
    TcW<K> W;
    float mx = 0.f;
    for (int i = 0; i < K * K * K; ++i) {
        W.w[i] = w[i];
        mx = std::max(mx, std::fabs(w[i]));
    }
    int ex = 0;
    if (mx > 0.f && std::isfinite(mx)) std::frexp(mx, &ex);
    a.wexp = (mx > 0.f && std::isfinite(mx)) ? std::min(std::max(14 - ex, -100), 100) : 0;

    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    a.items_x = (job.nx + 8 * XT - 1) / (8 * XT);
    a.items_y = (job.ny + MROWS - 1) / MROWS;
    const long xy = static_cast<long>(a.items_x) * a.items_y;
    // enough z chunks for ~6 items per SM, but chunks of at least 8 r planes
    long chunks = std::max<long>(1, (6L * sms + xy - 1) / xy);
    chunks = std::min<long>(chunks, std::max(1, job.nz / std::max(8, 8 * C::R)));
    a.zchunk = static_cast<int>((job.nz + chunks - 1) / chunks);
    a.items_z = (job.nz + a.zchunk - 1) / a.zchunk;
    a.nitems = static_cast<int>(xy * a.items_z);

    alignas(64) CUtensorMap map;
    if (!encode_tensor_map_3d(&map, FMT_F32, job.src, job.nx, job.ny, job.nz, NCH * 8, C::ROWS, 1))
        return VKT_ERROR_UNSUPPORTED;
    cudaError_t e = cudaFuncSetAttribute(k_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return from_cuda(e);
    const int grid = static_cast<int>(std::min<long>(a.nitems, sms));
    if (ctx.debug & VKT_DEBUG_LOG)
        fprintf(stderr, "[vkt] tensor k=%d items=%d (%dx%dx%d, zchunk %d) grid=%d smem=%d\n", K,
                a.nitems, a.items_x, a.items_y, a.items_z, a.zchunk, grid, C::SMEM);
    k_tc<K><<<grid, NTHREADS, C::SMEM, ctx.stream>>>(map, a, W);
    count_launches(1);
    return from_cuda(cudaGetLastError());
}

}  // namespace

vktError tensor_available(const vktStructuredVolume_impl* dst, const vktStructuredVolume_impl* src,
                          const vktFilter_impl* f)
{
    if (src->format != vktDataFormatFloat32 || dst->format != vktDataFormatFloat32)
        return VKT_ERROR_UNSUPPORTED;
    if (f->k != 5 && f->k != 7 && f->k != 9) return VKT_ERROR_UNSUPPORTED;
    if (src->dims[0] % 4 != 0 || reinterpret_cast<uintptr_t>(src->data) % 16 != 0)
        return VKT_ERROR_UNSUPPORTED;   // rows must be describable by a TMA tensor map
    return VKT_NO_ERROR;
}

vktError launch_tensor(const Job& job, const float* w, int k, const Ctx& ctx)
{
    switch (k) {
    case 5: return launch_k<5>(job, w, ctx);
    case 7: return launch_k<7>(job, w, ctx);
    case 9: return launch_k<9>(job, w, ctx);
    default: return VKT_ERROR_UNSUPPORTED;
    }
}

}  // namespace vkt
