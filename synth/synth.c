/*
 * synth.c -- seeded synthetic inputs shared by the GPU tests, the benchmark and the
 * oracle checks.  This file holds no filter arithmetic: it only draws volumes and
 * weights.  Every draw is counter based, so any element can be regenerated from
 * (seed, stream, index) alone, on any machine, in any thread order.
 *
 * Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), used as a hash of a 64-bit counter.
 * Normals: Box-Muller on two independent uniforms.
 *
 * Volumes are stored x fastest, then y, then z, matching the dims order of the
 * structured-volume create call (Sec. 3.2, Fig. exampleCvsCPP).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static inline uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* key of one (seed, stream) pair; each stream is an independent sequence */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream)
{
    return mix64(mix64(seed) ^ (stream * 0xD1B54A32D192ED03ull));
}

static inline uint64_t draw_u64(uint64_t key, uint64_t i)
{
    return mix64(key + i * 0x9E3779B97F4A7C15ull);
}

/* uniform in [0,1) with 53 random bits */
static inline double draw_u01(uint64_t key, uint64_t i)
{
    return (double)(draw_u64(key, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* standard normal from counters 2i and 2i+1 */
static inline double draw_normal(uint64_t key, uint64_t i)
{
    double u1 = 1.0 - draw_u01(key, 2 * i);     /* (0,1] so the log is finite */
    double u2 = draw_u01(key, 2 * i + 1);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

uint64_t synth_u64(uint64_t seed, uint64_t stream, uint64_t i)
{
    return draw_u64(stream_key(seed, stream), i);
}

double synth_u01(uint64_t seed, uint64_t stream, uint64_t i)
{
    return draw_u01(stream_key(seed, stream), i);
}

double synth_normal(uint64_t seed, uint64_t stream, uint64_t i)
{
    return draw_normal(stream_key(seed, stream), i);
}

void synth_uniform_f32(uint64_t seed, uint64_t stream, int64_t n, float lo, float hi, float* out)
{
    uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        out[i] = (float)(lo + (hi - lo) * draw_u01(key, (uint64_t)i));
}

void synth_normal_f32(uint64_t seed, uint64_t stream, int64_t n, double mean, double sd, float* out)
{
    uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        out[i] = (float)(mean + sd * draw_normal(key, (uint64_t)i));
}

/*
 * CT-like field: sum of nblobs isotropic Gaussian blobs (centres uniform in the volume,
 * sigma uniform in [smin,smax] voxels, amplitude uniform in [amin,amax]) plus i.i.d.
 * N(0,noise) per voxel, clamped to [0,1].  Blob parameters come from stream 1 of the
 * seed, the noise from stream 2.  Blobs are separable, so each one is the outer product
 * of three 1-D profiles, tabulated once.
 */
int synth_blobs_f32(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int nblobs,
                    double smin, double smax, double amin, double amax, double noise,
                    float* out)
{
    if (nblobs <= 0 || nblobs > 4096 || nx <= 0 || ny <= 0 || nz <= 0) return -1;
    double* tx = (double*)malloc(sizeof(double) * (size_t)nblobs * (size_t)(nx + ny + nz));
    if (!tx) return -2;
    double* ty = tx + (size_t)nblobs * nx;
    double* tz = ty + (size_t)nblobs * ny;
    uint64_t kp = stream_key(seed, 1), kn = stream_key(seed, 2);
    for (int b = 0; b < nblobs; ++b) {
        double cx = draw_u01(kp, 5 * b + 0) * (double)nx;
        double cy = draw_u01(kp, 5 * b + 1) * (double)ny;
        double cz = draw_u01(kp, 5 * b + 2) * (double)nz;
        double sg = smin + (smax - smin) * draw_u01(kp, 5 * b + 3);
        double am = amin + (amax - amin) * draw_u01(kp, 5 * b + 4);
        double inv = 1.0 / (2.0 * sg * sg);
        for (int64_t x = 0; x < nx; ++x) { double d = x - cx; tx[b * nx + x] = exp(-d * d * inv); }
        for (int64_t y = 0; y < ny; ++y) { double d = y - cy; ty[b * ny + y] = exp(-d * d * inv); }
        for (int64_t z = 0; z < nz; ++z) { double d = z - cz; tz[b * nz + z] = am * exp(-d * d * inv); }
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|:bad)
    for (int64_t z = 0; z < nz; ++z) {
        double* acc = (double*)malloc(sizeof(double) * (size_t)nx);
        if (!acc) { bad = 1; continue; }
        for (int64_t y = 0; y < ny; ++y) {
            for (int64_t x = 0; x < nx; ++x) acc[x] = 0.0;
            for (int b = 0; b < nblobs; ++b) {
                double fyz = tz[b * nz + z] * ty[b * ny + y];
                const double* g = tx + (size_t)b * nx;
                for (int64_t x = 0; x < nx; ++x) acc[x] += fyz * g[x];
            }
            int64_t base = (z * ny + y) * nx;
            for (int64_t x = 0; x < nx; ++x) {
                double v = acc[x] + noise * draw_normal(kn, (uint64_t)(base + x));
                v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
                out[base + x] = (float)v;
            }
        }
        free(acc);
    }
    free(tx);
    return bad ? -2 : 0;
}

/* quantise values in [0,1] to unsigned codes of `bits` bits: q = floor(v*(2^bits-1) + 1/2) */
void synth_quantize(const float* v, int64_t n, int bits, void* out)
{
    double qmax = (double)((1u << bits) - 1u);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double t = floor((double)v[i] * qmax + 0.5);
        t = t < 0.0 ? 0.0 : (t > qmax ? qmax : t);
        if (bits == 8) ((uint8_t*)out)[i] = (uint8_t)t;
        else ((uint16_t*)out)[i] = (uint16_t)t;
    }
}

/*
 * Simulation-like field: sum of nmodes Fourier modes.  Mode m has wavenumber magnitude
 * |k| uniform in [kmin,kmax] cycles per domain, direction uniform on the sphere, phase
 * uniform in [0,2pi) and amplitude |k|^(-5/3):
 *     f(x,y,z) = sum_m a_m cos(2 pi (kx x/nx + ky y/ny + kz z/nz) + phi_m).
 * Mode parameters come from stream 3.  Evaluated as Re(a e^{i phi} e^{i B(y)} e^{i C(z)}
 * e^{i A(x)}) with the x factors tabulated once, so each voxel costs two multiply-adds
 * per mode.
 */
int synth_fourier_f32(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int nmodes,
                      double kmin, double kmax, float* out)
{
    if (nmodes <= 0 || nmodes > 1024 || nx <= 0 || ny <= 0 || nz <= 0) return -1;
    double par[5 * 1024];
    uint64_t km = stream_key(seed, 3);
    double* ex = (double*)malloc(sizeof(double) * 2 * (size_t)nmodes * (size_t)nx);
    if (!ex) return -2;
    for (int m = 0; m < nmodes; ++m) {
        double kk = kmin + (kmax - kmin) * draw_u01(km, 5 * m + 0);
        double cz = 2.0 * draw_u01(km, 5 * m + 1) - 1.0;
        double az = 2.0 * M_PI * draw_u01(km, 5 * m + 2);
        double sz = sqrt(1.0 - cz * cz);
        par[5 * m + 0] = kk * sz * cos(az);   /* kx */
        par[5 * m + 1] = kk * sz * sin(az);   /* ky */
        par[5 * m + 2] = kk * cz;             /* kz */
        par[5 * m + 3] = 2.0 * M_PI * draw_u01(km, 5 * m + 3);
        par[5 * m + 4] = pow(kk, -5.0 / 3.0);
        double wx = 2.0 * M_PI * par[5 * m + 0] / (double)nx;
        for (int64_t x = 0; x < nx; ++x) {
            ex[(2 * (size_t)m) * nx + x] = cos(wx * (double)x);
            ex[(2 * (size_t)m + 1) * nx + x] = sin(wx * (double)x);
        }
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|:bad)
    for (int64_t z = 0; z < nz; ++z) {
        double* acc = (double*)malloc(sizeof(double) * (size_t)nx);
        if (!acc) { bad = 1; continue; }
        for (int64_t y = 0; y < ny; ++y) {
            for (int64_t x = 0; x < nx; ++x) acc[x] = 0.0;
            for (int m = 0; m < nmodes; ++m) {
                double phase = 2.0 * M_PI * (par[5 * m + 1] * (double)y / (double)ny +
                                             par[5 * m + 2] * (double)z / (double)nz) +
                               par[5 * m + 3];
                double cr = par[5 * m + 4] * cos(phase), ci = par[5 * m + 4] * sin(phase);
                const double* er = ex + (2 * (size_t)m) * nx;
                const double* ei = er + nx;
                for (int64_t x = 0; x < nx; ++x) acc[x] += cr * er[x] - ci * ei[x];
            }
            int64_t base = (z * ny + y) * nx;
            for (int64_t x = 0; x < nx; ++x) out[base + x] = (float)acc[x];
        }
        free(acc);
    }
    free(ex);
    return bad ? -2 : 0;
}
