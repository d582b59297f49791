/*
 * oracle.c -- plain FP64 CPU reference for ApplyFilter.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg call this code.  It shares no code with the CUDA library and includes
 * none of its headers.
 *
 * What is computed (Sec. 3.2, "Volume Manipulation"): ApplyFilter applies a
 * user-specified convolution kernel (edge detection, Gaussian blur) to a structured
 * volume, with the same result as the per-cell formulation through Transform.  The
 * paper fixes no boundary rule, no anchor and no index order, so this file takes these
 * readings:
 *   - correlation form, anchor at the kernel centre r = (k-1)/2, k odd:
 *       y(x,y,z) = sum_{a,b,c in [-r,r]} w[c+r][b+r][a+r] * v(X(x+a), Y(y+b), Z(z+c))
 *   - clamp-to-edge boundary: X(i) = min(max(i,0), nx-1), same for Y and Z;
 *   - memory order x fastest, then y, then z (dims order of the create call, Fig.
 *     exampleCvsCPP); weights stored the same way, a fastest;
 *   - value mapping of a stored voxel q (Sec. 3.2, create call with format and range):
 *       uint8/uint16: v = lo + (hi - lo) * q / (2^N - 1);   float32: v = q;
 *   - quantisation to an integer destination:
 *       t = (v - lo)/(hi - lo) * (2^N - 1),  q = clamp(round-half-even(t), 0, 2^N - 1).
 * Everything is evaluated in double precision, one voxel at a time, taps in order.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <fenv.h>

enum { OR_U8 = 0, OR_U16 = 1, OR_F32 = 2 };

static int64_t clampi(int64_t i, int64_t n)
{
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

/* value of stored voxel number i under the volume's mapping range [lo,hi] */
static double mapped(const void* src, int fmt, int64_t i, double lo, double hi)
{
    switch (fmt) {
    case OR_U8:  return lo + (hi - lo) * (double)((const uint8_t*)src)[i] / 255.0;
    case OR_U16: return lo + (hi - lo) * (double)((const uint16_t*)src)[i] / 65535.0;
    default:     return (double)((const float*)src)[i];
    }
}

static int check_args(int fmt, int64_t nx, int64_t ny, int64_t nz, int k)
{
    if (fmt < OR_U8 || fmt > OR_F32) return -1;
    if (nx < 0 || ny < 0 || nz < 0) return -1;
    if (k < 1 || (k & 1) == 0) return -1;
    return 0;
}

/* one output voxel, straight from the definition above */
static double correlate_at(const void* src, int fmt, double lo, double hi,
                           int64_t nx, int64_t ny, int64_t nz, const double* w, int k,
                           int64_t x, int64_t y, int64_t z)
{
    int r = (k - 1) / 2;
    double acc = 0.0;
    for (int c = 0; c < k; ++c) {
        int64_t zz = clampi(z + c - r, nz);
        for (int b = 0; b < k; ++b) {
            int64_t yy = clampi(y + b - r, ny);
            for (int a = 0; a < k; ++a) {
                int64_t xx = clampi(x + a - r, nx);
                acc += w[((int64_t)c * k + b) * k + a] *
                       mapped(src, fmt, (zz * ny + yy) * nx + xx, lo, hi);
            }
        }
    }
    return acc;
}

/* full volume: out[(z*ny + y)*nx + x] = y(x,y,z) as a double */
int oracle_correlate(const void* src, int fmt, double lo, double hi,
                     int64_t nx, int64_t ny, int64_t nz, const double* w, int k,
                     double* out)
{
    if (check_args(fmt, nx, ny, nz, k)) return -1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x)
                out[(z * ny + y) * nx + x] =
                    correlate_at(src, fmt, lo, hi, nx, ny, nz, w, k, x, y, z);
    return 0;
}

/* selected voxels only (linear indices), for checks at sizes the full loop cannot reach */
int oracle_correlate_points(const void* src, int fmt, double lo, double hi,
                            int64_t nx, int64_t ny, int64_t nz, const double* w, int k,
                            const int64_t* idx, int64_t npts, double* out)
{
    if (check_args(fmt, nx, ny, nz, k)) return -1;
    int64_t nvox = nx * ny * nz;
    for (int64_t p = 0; p < npts; ++p)
        if (idx[p] < 0 || idx[p] >= nvox) return -2;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npts; ++p) {
        int64_t i = idx[p];
        int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
        out[p] = correlate_at(src, fmt, lo, hi, nx, ny, nz, w, k, x, y, z);
    }
    return 0;
}

/*
 * Quantisation of filtered values to an integer destination with range [lo,hi]
 * (bits = 8 or 16).  t[i] receives the pre-rounding code value, q[i] the code, and
 * tie[i] = 1 where t lies within `window` of a half-integer (there either neighbour is
 * accepted, since no precision short of exact arithmetic decides it).
 */
int oracle_quantize(const double* v, int64_t n, int bits, double lo, double hi,
                    double window, double* t, uint32_t* q, uint8_t* tie)
{
    if ((bits != 8 && bits != 16) || !(hi != lo)) return -1;
    double qmax = (double)((1u << bits) - 1u);
    int old = fegetround();
    fesetround(FE_TONEAREST);
    for (int64_t i = 0; i < n; ++i) {
        double ti = (v[i] - lo) / (hi - lo) * qmax;
        double qi = ti != ti ? 0.0 : nearbyint(ti);   /* NaN reads as 0 */
        qi = qi < 0.0 ? 0.0 : (qi > qmax ? qmax : qi);
        t[i] = ti;
        q[i] = (uint32_t)qi;
        tie[i] = (uint8_t)(fabs(ti - floor(ti) - 0.5) < window);
    }
    fesetround(old);
    return 0;
}

/*
 * Filter construction (Gaussian blur, Sec. 1 teaser and Sec. 4.3).  The paper gives
 * neither size nor sigma, and no definition beyond "Gaussian blur"; the reading taken:
 * the sampled Gaussian g(d) = exp(-d^2 / (2 sigma^2)) at the integer offsets
 * d in [-r, r], divided by its sum (FP64), stored as float32.  The 3-D kernel is the
 * product g[c]*g[b]*g[a] of the stored 1-D weights (the sampled 3-D Gaussian factorises
 * exactly, so this is the sampled 3-D Gaussian normalised to sum 1).
 */
int oracle_gaussian_1d(int k, double sigma, float* g)
{
    if (k < 1 || (k & 1) == 0 || !(sigma > 0.0)) return -1;
    int r = (k - 1) / 2;
    double e[64], s = 0.0;
    if (k > 63) return -1;
    for (int i = 0; i < k; ++i) {
        double d = (double)(i - r);
        e[i] = exp(-d * d / (2.0 * sigma * sigma));
        s += e[i];
    }
    for (int i = 0; i < k; ++i) g[i] = (float)(e[i] / s);
    return 0;
}

/* dense k^3 weights (double) of a separable filter: w[c][b][a] = gz[c] * gy[b] * gx[a] */
void oracle_separable_weights(int k, const float* gx, const float* gy, const float* gz,
                              double* w)
{
    for (int c = 0; c < k; ++c)
        for (int b = 0; b < k; ++b)
            for (int a = 0; a < k; ++a)
                w[((int64_t)c * k + b) * k + a] = (double)gz[c] * (double)gy[b] * (double)gx[a];
}

/*
 * Gradients of the float32 filter y = C_w x (x float-valued, identity mapping), for a
 * loss L with dL/dy = gy.  Straight from the definition of y above:
 *   gx[j] = sum_i sum_d w[d] gy[i] [clamp(i+d) == j]      (adjoint, scatter form)
 *   gw[d] = sum_i gy[i] x[clamp(i+d)]
 * The scatter is serial: each input voxel receives from every tap whose clamped
 * position lands on it, which at a face includes several taps of the same output.
 */
int oracle_correlate_backward(const double* x, const double* gy, int64_t nx, int64_t ny,
                              int64_t nz, const double* w, int k, double* gx, double* gw)
{
    if (check_args(OR_F32, nx, ny, nz, k)) return -1;
    int r = (k - 1) / 2;
    int64_t n = nx * ny * nz;
    if (gx) {
        memset(gx, 0, sizeof(double) * (size_t)n);
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t xx = 0; xx < nx; ++xx) {
                    double g = gy[(z * ny + y) * nx + xx];
                    for (int c = 0; c < k; ++c) {
                        int64_t sz = clampi(z + c - r, nz);
                        for (int b = 0; b < k; ++b) {
                            int64_t sy = clampi(y + b - r, ny);
                            for (int a = 0; a < k; ++a) {
                                int64_t sx = clampi(xx + a - r, nx);
                                gx[(sz * ny + sy) * nx + sx] += w[((int64_t)c * k + b) * k + a] * g;
                            }
                        }
                    }
                }
    }
    if (gw) {
        int64_t kk = (int64_t)k * k * k;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t d = 0; d < kk; ++d) {
            int a = (int)(d % k), b = (int)((d / k) % k), c = (int)(d / ((int64_t)k * k));
            double acc = 0.0;
            for (int64_t z = 0; z < nz; ++z) {
                int64_t sz = clampi(z + c - r, nz);
                for (int64_t y = 0; y < ny; ++y) {
                    int64_t sy = clampi(y + b - r, ny);
                    for (int64_t xx = 0; xx < nx; ++xx) {
                        int64_t sx = clampi(xx + a - r, nx);
                        acc += gy[(z * ny + y) * nx + xx] * x[(sz * ny + sy) * nx + sx];
                    }
                }
            }
            gw[d] = acc;
        }
    }
    return 0;
}

/*
 * gx at selected voxels j, from the same definition: the outputs i that reach j through
 * tap d are those whose clamped position i+d equals j on every axis.  Per axis (n > 1):
 * j interior -> i = j - d (if in range); j = 0 -> every i with i + d <= 0;
 * j = n-1 -> every i with i + d >= n-1.  (n = 1: every i, i.e. i = 0.)
 */
static void axis_sources(int64_t j, int d, int64_t n, int64_t* i0, int64_t* i1)
{
    int64_t lo, hi;
    if (n == 1) { lo = 0; hi = 0; }
    else if (j == 0) { lo = 0; hi = -d; }
    else if (j == n - 1) { lo = n - 1 - d; hi = n - 1; }
    else { lo = j - d; hi = j - d; }
    if (lo < 0) lo = 0;
    if (hi > n - 1) hi = n - 1;
    *i0 = lo;
    *i1 = hi;   /* empty when lo > hi */
}

int oracle_backward_input_points(const double* gy, int64_t nx, int64_t ny, int64_t nz,
                                 const double* w, int k, const int64_t* idx, int64_t npts,
                                 double* out)
{
    if (check_args(OR_F32, nx, ny, nz, k)) return -1;
    int r = (k - 1) / 2;
    int64_t nvox = nx * ny * nz;
    for (int64_t p = 0; p < npts; ++p)
        if (idx[p] < 0 || idx[p] >= nvox) return -2;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npts; ++p) {
        int64_t j = idx[p];
        int64_t jx = j % nx, jy = (j / nx) % ny, jz = j / (nx * ny);
        double acc = 0.0;
        for (int c = 0; c < k; ++c) {
            int64_t z0, z1;
            axis_sources(jz, c - r, nz, &z0, &z1);
            for (int b = 0; b < k; ++b) {
                int64_t y0, y1;
                axis_sources(jy, b - r, ny, &y0, &y1);
                for (int a = 0; a < k; ++a) {
                    int64_t x0, x1;
                    axis_sources(jx, a - r, nx, &x0, &x1);
                    double wd = w[((int64_t)c * k + b) * k + a];
                    for (int64_t z = z0; z <= z1; ++z)
                        for (int64_t y = y0; y <= y1; ++y)
                            for (int64_t x = x0; x <= x1; ++x)
                                acc += wd * gy[(z * ny + y) * nx + x];
                }
            }
        }
        out[p] = acc;
    }
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops over output voxels (timing only; results do not depend on
 * it: every voxel's sum is evaluated by one thread in the definition's tap order). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/*
 * CLAHE-3D (Sec. 4.1 "Case Study: CLAHE-3D": contrast limited adaptive histogram
 * equalisation, a 3-D variant of the 2-D method; brick decomposition, local histograms, a
 * maximum cut-off on the histograms, and linear interpolation of the local results).  The
 * paper gives the steps but not their constants; the readings taken (uint8 volumes):
 *   - bricks: nb = (nbx, nby, nbz) bricks per axis that divide the dims exactly; brick size
 *     s = dims / nb, N = sx*sy*sz voxels per brick;
 *   - histogram: 256 bins of the stored codes of each brick;
 *   - clip: limit L = max(1, floor(clip * N / 256)) (clip <= 0: no clipping); the excess
 *     E = sum max(h - L, 0) is removed and given back evenly, E / 256 to every bin, and the
 *     remaining E mod 256 counts one each to bins 0, step, 2 step, ... with
 *     step = max(1, 256 / (E mod 256)), while any remain;
 *   - mapping of a brick: lut[q] = floor((255 * cdf[q] + N / 2) / N), cdf[q] = sum_{i<=q} h[i];
 *   - interpolation: voxel x lies at brick coordinate t = (x + 0.5) / sx - 0.5 per axis;
 *     b0 = floor(t), w = t - b0, b1 = b0 + 1, both clamped to [0, nb - 1]; the result is the
 *     trilinear blend of the 8 bricks' lut[q] with weights (1 - w, w) per axis, rounded
 *     half-to-even to a code.
 * t_out receives the blended values before rounding (for the tie window of the tests).
 */
static void clahe_lut(const int64_t* hist_in, int64_t n, double clip, uint8_t* lut)
{
    int64_t h[256];
    for (int i = 0; i < 256; ++i) h[i] = hist_in[i];
    if (clip > 0.0) {
        int64_t limit = (int64_t)floor(clip * (double)n / 256.0);
        if (limit < 1) limit = 1;
        int64_t excess = 0;
        for (int i = 0; i < 256; ++i)
            if (h[i] > limit) {
                excess += h[i] - limit;
                h[i] = limit;
            }
        const int64_t add = excess / 256;
        int64_t rem = excess - add * 256;
        for (int i = 0; i < 256; ++i) h[i] += add;
        if (rem > 0) {
            int64_t step = 256 / rem;
            if (step < 1) step = 1;
            for (int64_t i = 0; i < 256 && rem > 0; i += step) {
                h[i] += 1;
                rem -= 1;
            }
        }
    }
    int64_t cdf = 0;
    for (int i = 0; i < 256; ++i) {
        cdf += h[i];
        int64_t v = (255 * cdf + n / 2) / n;
        lut[i] = (uint8_t)(v > 255 ? 255 : v);
    }
}

int oracle_clahe3d(const uint8_t* src, int64_t nx, int64_t ny, int64_t nz, int nbx, int nby,
                   int nbz, double clip, uint8_t* out, double* t_out, uint8_t* luts_out)
{
    if (nbx < 1 || nby < 1 || nbz < 1) return -1;
    if (nx % nbx || ny % nby || nz % nbz) return -1;
    const int64_t sx = nx / nbx, sy = ny / nby, sz = nz / nbz, n = sx * sy * sz;
    const int64_t nbricks = (int64_t)nbx * nby * nbz;
    uint8_t* luts = (uint8_t*)malloc((size_t)nbricks * 256);
    int64_t* hist = (int64_t*)calloc((size_t)nbricks * 256, sizeof(int64_t));
    if (!luts || !hist) {
        free(luts);
        free(hist);
        return -2;
    }
    /* local histograms */
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t b = ((z / sz) * nby + (y / sy)) * nbx + (x / sx);
                hist[b * 256 + src[(z * ny + y) * nx + x]] += 1;
            }
    /* clipped, redistributed, equalised mapping of every brick */
    for (int64_t b = 0; b < nbricks; ++b) clahe_lut(hist + b * 256, n, clip, luts + b * 256);
    /* trilinear blend of the 8 nearest bricks' mappings */
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z) {
        const double tz = ((double)z + 0.5) / (double)sz - 0.5;
        const double fz = floor(tz), wz = tz - fz;
        const int64_t z0 = clampi((int64_t)fz, nbz), z1 = clampi((int64_t)fz + 1, nbz);
        for (int64_t y = 0; y < ny; ++y) {
            const double ty = ((double)y + 0.5) / (double)sy - 0.5;
            const double fy = floor(ty), wy = ty - fy;
            const int64_t y0 = clampi((int64_t)fy, nby), y1 = clampi((int64_t)fy + 1, nby);
            for (int64_t x = 0; x < nx; ++x) {
                const double tx = ((double)x + 0.5) / (double)sx - 0.5;
                const double fx = floor(tx), wx = tx - fx;
                const int64_t x0 = clampi((int64_t)fx, nbx), x1 = clampi((int64_t)fx + 1, nbx);
                const int64_t i = (z * ny + y) * nx + x;
                const int q = src[i];
                double v = 0.0;
                for (int c = 0; c < 8; ++c) {
                    const int64_t bx = (c & 1) ? x1 : x0, by = (c & 2) ? y1 : y0, bz = (c & 4) ? z1 : z0;
                    const double w = ((c & 1) ? wx : 1.0 - wx) * ((c & 2) ? wy : 1.0 - wy) *
                                     ((c & 4) ? wz : 1.0 - wz);
                    v += w * (double)luts[((bz * nby + by) * nbx + bx) * 256 + q];
                }
                if (t_out) t_out[i] = v;
                double r = nearbyint(v);     /* round half to even (default rounding mode) */
                out[i] = (uint8_t)(r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r));
            }
        }
    }
    if (luts_out) memcpy(luts_out, luts, (size_t)nbricks * 256);
    free(luts);
    free(hist);
    return 0;
}

/*
 * Headless Render, ray marching with absorption and emission (Sec. 3.2 "Rendering": the
 * Render algorithm's volume ray marching with absorption and emission, classified by an
 * RGBA lookup table).  No window: one RGBA value per pixel.  Readings (the paper gives
 * none of these):
 *   - world = voxel units, the volume is the box [0,nx] x [0,ny] x [0,nz], voxel (i,j,k)
 *     centred at (i+0.5, j+0.5, k+0.5); a sample's value is the trilinear blend of the
 *     mapped voxel values at p - 0.5 (indices clamped to the volume);
 *   - classification: u = clamp((v - lo) / (hi - lo), 0, 1); the table's n entries sit at
 *     u = i / (n-1) and are blended linearly; colours are straight (not premultiplied),
 *     alpha is the opacity of one voxel length and is corrected to the step:
 *     a' = 1 - (1 - a)^step;
 *   - camera: pinhole at eye looking at center, vertical field of view fovy, up vector;
 *     pixel (px, py) (py = 0 at the top) looks along
 *       normalize(f + (2(px+0.5)/W - 1) tan(fovy/2) (W/H) r + (1 - 2(py+0.5)/H) tan(fovy/2) u),
 *     f = normalize(center - eye), r = normalize(f x up), u = r x f;
 *   - the ray enters the box at t0 = max(tnear, 0), leaves at t1 (slab test; an axis with a
 *     direction component below 1e-12 in magnitude is parallel: the ray misses the box if it
 *     lies outside that slab); samples at t0 + (k + 0.5) step while below t1;
 *   - front-to-back compositing: C += (1 - A) a' c, A += (1 - A) a'; marching stops after a
 *     sample that brings A to `termination` or above;
 *   - pixel = (C + (1 - A) bg.rgb, A + (1 - A) bg.a).
 */
static double sample_trilinear(const void* src, int fmt, double lo, double hi, int64_t nx,
                               int64_t ny, int64_t nz, double px, double py, double pz)
{
    const double x = px - 0.5, y = py - 0.5, z = pz - 0.5;
    const double fx = floor(x), fy = floor(y), fz = floor(z);
    const double wx = x - fx, wy = y - fy, wz = z - fz;
    const int64_t ix = (int64_t)fx, iy = (int64_t)fy, iz = (int64_t)fz;
    double v = 0.0;
    for (int c = 0; c < 8; ++c) {
        const int64_t i = clampi(ix + (c & 1), nx), j = clampi(iy + ((c >> 1) & 1), ny),
                      k = clampi(iz + ((c >> 2) & 1), nz);
        const double w = ((c & 1) ? wx : 1.0 - wx) * (((c >> 1) & 1) ? wy : 1.0 - wy) *
                         (((c >> 2) & 1) ? wz : 1.0 - wz);
        v += w * mapped(src, fmt, (k * ny + j) * nx + i, lo, hi);
    }
    return v;
}

static void normalize3(double* v)
{
    const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n;
    v[1] /= n;
    v[2] /= n;
}

/* the pixels listed in pix (npix (px, py) pairs; all pixels when pix is NULL) */
int oracle_render_pixels(const void* src, int fmt, double lo, double hi, int64_t nx, int64_t ny,
                         int64_t nz, int width, int height, const double* eye,
                         const double* center, const double* up, double fovy, double step,
                         double termination, const double* bg, int lut_n, const double* lut,
                         const int32_t* pix, int64_t npix, double* rgba);

int oracle_render(const void* src, int fmt, double lo, double hi, int64_t nx, int64_t ny,
                  int64_t nz, int width, int height, const double* eye, const double* center,
                  const double* up, double fovy, double step, double termination,
                  const double* bg, int lut_n, const double* lut, double* rgba)
{
    return oracle_render_pixels(src, fmt, lo, hi, nx, ny, nz, width, height, eye, center, up,
                                fovy, step, termination, bg, lut_n, lut, NULL,
                                (int64_t)width * height, rgba);
}

int oracle_render_pixels(const void* src, int fmt, double lo, double hi, int64_t nx, int64_t ny,
                         int64_t nz, int width, int height, const double* eye,
                         const double* center, const double* up, double fovy, double step,
                         double termination, const double* bg, int lut_n, const double* lut,
                         const int32_t* pix, int64_t npix, double* rgba)
{
    if (width < 1 || height < 1 || lut_n < 2 || !(step > 0.0)) return -1;
    double f[3] = {center[0] - eye[0], center[1] - eye[1], center[2] - eye[2]};
    normalize3(f);
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    normalize3(r);
    const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    const double th = tan(0.5 * fovy), aspect = (double)width / (double)height;
    const double box[3] = {(double)nx, (double)ny, (double)nz};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t n = 0; n < npix; ++n) {
            const int px = pix ? pix[2 * n] : (int)(n % width);
            const int py = pix ? pix[2 * n + 1] : (int)(n / width);
            const double sx = (2.0 * (px + 0.5) / width - 1.0) * th * aspect;
            const double sy = (1.0 - 2.0 * (py + 0.5) / height) * th;
            double d[3] = {f[0] + sx * r[0] + sy * u[0], f[1] + sx * r[1] + sy * u[1],
                           f[2] + sx * r[2] + sy * u[2]};
            normalize3(d);
            double tn = -INFINITY, tf = INFINITY;
            int hit = 1;
            for (int a = 0; a < 3; ++a) {
                if (fabs(d[a]) < 1e-12) {
                    if (eye[a] < 0.0 || eye[a] > box[a]) hit = 0;
                    continue;
                }
                double ta = (0.0 - eye[a]) / d[a], tb = (box[a] - eye[a]) / d[a];
                if (ta > tb) {
                    const double t = ta;
                    ta = tb;
                    tb = t;
                }
                if (ta > tn) tn = ta;
                if (tb < tf) tf = tb;
            }
            const double t0 = tn > 0.0 ? tn : 0.0, t1 = tf;
            double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
            if (hit && t0 < t1) {
                for (int64_t k = 0;; ++k) {
                    const double t = t0 + ((double)k + 0.5) * step;
                    if (!(t < t1)) break;
                    const double v = sample_trilinear(src, fmt, lo, hi, nx, ny, nz, eye[0] + t * d[0],
                                                      eye[1] + t * d[1], eye[2] + t * d[2]);
                    double un = (v - lo) / (hi - lo);
                    un = un < 0.0 ? 0.0 : (un > 1.0 ? 1.0 : un);
                    const double fi = un * (lut_n - 1);
                    int i0 = (int)floor(fi);
                    if (i0 > lut_n - 2) i0 = lut_n - 2;
                    const double w = fi - i0;
                    double c[4];
                    for (int ch = 0; ch < 4; ++ch)
                        c[ch] = (1.0 - w) * lut[4 * i0 + ch] + w * lut[4 * (i0 + 1) + ch];
                    const double ac = 1.0 - pow(1.0 - c[3], step);
                    for (int ch = 0; ch < 3; ++ch) C[ch] += (1.0 - A) * ac * c[ch];
                    A += (1.0 - A) * ac;
                    if (A >= termination) break;
                }
            }
            double* o = rgba + 4 * (pix ? n : ((int64_t)py * width + px));
            for (int ch = 0; ch < 3; ++ch) o[ch] = C[ch] + (1.0 - A) * bg[ch];
            o[3] = A + (1.0 - A) * bg[3];
        }
    return 0;
}
