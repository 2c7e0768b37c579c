/*
 * pgrec: seeded synthetic scenes and an instrumented volumetric path tracer
 * that records path-graph inputs.
 *
 * This is the input generator shared by the FP64 oracle and the CUDA path.
 * It plays the role of the paper's instrumented path tracer (Section 4,
 * "Instrumented path tracer"; Section 3.4 "Volume Path Tracing"): it traces
 * camera paths through a voxel medium with delta tracking, takes one emitter
 * (next-event) sample and one phase-function sample at every scattering
 * vertex, and records every vertex in one global array in path order.
 *
 * It computes its own path-tracing estimate (the image and, per vertex, the
 * incoming indirect radiance along the phase-sampled direction) the way a
 * path tracer does, by walking each path; it does not evaluate any
 * path-graph aggregation or propagation operator.
 *
 * Conventions (all directions unit length):
 *   o_v  direction from x_v toward the previous vertex (or the camera)
 *   d_v  phase-sampled direction at x_v (light arrives from x_v + t d_v)
 *   e_v  emitter-sample direction at x_v
 *   Henyey-Greenstein phase with mu = -o.d, so g > 0 scatters forward.
 * Light model: an optional directional "sun" (a delta light, sampled with
 * probability p_sun) and continuous emitters (a constant environment and an
 * optional one-sided rectangular area light), treated together as one
 * emitter-sampling strategy whose pdf is the selection-weighted mixture.
 * The area light does not occlude the environment (their radiance adds).
 *
 * Randomness: every path draws from its own counter-based splitmix64 stream
 * keyed by (seed, path index), so the output does not depend on the number
 * of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_D 3.14159265358979323846
#define PG_INV_4PI 0.07957746833562851f /* 1/(4 pi), float */

typedef struct {
    /* medium: [0,1]^3 voxel grid, nearest-voxel lookup */
    int32_t grid_res;       /* voxels per axis */
    int32_t medium_kind;    /* 0 = constant sigma_t, 1 = fBm cloud */
    float sigma_t_max;      /* constant value, or the cloud's maximum */
    float albedo;           /* used when no albedo grid is given */
    float g;                /* Henyey-Greenstein asymmetry */
    int32_t fbm_octaves;
    float fbm_base_freq;
    float fbm_lacunarity;
    float fbm_gain;
    float cloud_threshold;  /* fBm level mapped to zero density */
    float cloud_radius;     /* spherical falloff radius around (0.5,0.5,0.5) */
    uint64_t seed;
    /* lights */
    float sun_dir[3];       /* direction the sunlight travels */
    float sun_irradiance;   /* 0 = no sun */
    float sky_radiance;     /* constant environment, 0 = none */
    float area_radiance;    /* 0 = no area light */
    float area_center[3];
    float area_u[3];        /* half-edge vectors; emits toward +(u x v) */
    float area_v[3];
    float p_sun;            /* probability of picking the sun in NEE */
    float p_area;           /* share of the area light among continuous lights */
    /* camera */
    int32_t width, height, spp, max_depth;
    float cam_pos[3];
    float cam_target[3];
    float cam_fov_deg;      /* vertical field of view */
    int32_t extra_direct;   /* extra emitter samples recorded at each path's first
                               vertex (Section 4, "Handling direct light"); 0 = none */
} pgrec_config;

typedef struct {
    /* per-thread growable vertex buffers */
    int64_t n, cap;
    float *px, *py, *pz, *ox, *oy, *oz, *dx, *dy, *dz, *ex, *ey, *ez;
    float *g, *sigma_s, *sigma_t, *w_prop, *Le, *pe_e, *Lph, *pe_ph, *L0;
    double *L0_f64;
    uint8_t *e_delta;
    int32_t *succ_local; /* -1 or offset within the path */
    int32_t *voxel;
} vbuf;

typedef struct {
    pgrec_config cfg;
    float *density;      /* grid_res^3 sigma_t */
    float *albedo_grid;  /* grid_res^3 albedo */
    int64_t n_paths;
    int nthreads;
    vbuf *bufs;
    int64_t *path_first_local; /* per path: local vertex index in its thread buffer or -1 */
    int32_t *path_thread;
    float *bg;
    double *val;
    float *x_e;          /* n_paths * extra_direct * 3 extra emitter-sample directions */
    float *x_Le, *x_pe;  /* their radiance and pdf (as Le / pe_e of a vertex) */
    uint8_t *x_delta;    /* 1 for a delta-light sample */
    int64_t n_vertices;
    int64_t *thread_offset;
    float majorant;      /* max sigma_t over the grid (delta-tracking bound) */
    float p_sun;         /* probability that the emitter sample picks the sun */
    float tan_half_fov;  /* tan of half the vertical field of view */
} pgrec_state;

/* ---------------- random numbers ---------------- */
typedef struct { uint64_t s; } rng_t;
static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* uniform on [0, 1) with 24 random bits (exact in float) */
static inline float rnd(rng_t *r) {
    r->s += 0x9E3779B97F4A7C15ULL;
    return (float)(mix64(r->s) >> 40) * (1.0f / 16777216.0f);
}

/* ---------------- elementary functions ----------------
 * The path tracing runs in single precision with its own logarithm and
 * sin/cos (rather than the C library's), built without FMA contraction, so
 * that the GPU recorder, which evaluates the same formulas in the same order,
 * produces bit-identical paths: both use only IEEE-rounded +, -, *, /, sqrt
 * and exact operations (frexp, floor, scaling by powers of two).
 *
 * pg_log: x = m 2^e with m in [1/sqrt2, sqrt2); log m = 2 artanh(s),
 * s = (m - 1)/(m + 1), |s| <= 0.1716, by its odd power series to s^11
 * (remainder below 1e-10); log x = e ln2 + log m with ln2 split into a
 * 12-bit head (e * head exact) and a tail. */
static const float PG_LN2_HI = 0.693115234375f, PG_LN2_LO = 3.194618329871446e-05f;
static const float PG_ATANH_C[5] = {0.3333333432674408f, 0.20000000298023224f, 0.1428571492433548f,
                                    0.1111111119389534f, 0.09090909361839294f}; /* 1/3, 1/5, ..., 1/11 */
static float pg_log(float x) {
    int e;
    float m = frexpf(x, &e);
    if (m < 0.7071067690849304f) {
        m = m * 2.0f;
        e = e - 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = PG_ATANH_C[4];
    for (int k = 3; k >= 0; k--) p = p * s2 + PG_ATANH_C[k];
    p = p * s2 + 1.0f;
    float lm = 2.0f * s * p;
    return (float)e * PG_LN2_HI + ((float)e * PG_LN2_LO + lm);
}

/* pg_sincos_2pi: sin and cos of 2 pi u for u in [0, 1). 4u = q + f
 * (quadrant q, f in [0, 1), both exact), a = f pi/2 in [0, pi/2), Taylor
 * series of sin a to a^13 and cos a to a^12 (remainder below 1e-8), then the
 * quadrant's symmetry. */
static const float PG_HALF_PI = 1.5707963705062866f;
static const float PG_SIN_C[6] = {-0.1666666716337204f, 0.008333333767950535f, -0.00019841270113829523f,
                                  2.7557318844628753e-06f, -2.5052107943679403e-08f,
                                  1.6059044372074283e-10f}; /* (-1)^k/(2k+1)! */
static const float PG_COS_C[6] = {-0.5f, 0.0416666679084301f, -0.0013888889225199819f, 2.4801587642286904e-05f,
                                  -2.755731998149713e-07f, 2.0876755879584152e-09f}; /* (-1)^k/(2k)! */
static void pg_sincos_2pi(float u, float *s_out, float *c_out) {
    float t = 4.0f * u;
    float q = floorf(t);
    float f = t - q;
    float a = f * PG_HALF_PI;
    float a2 = a * a;
    float ps = PG_SIN_C[5], pc = PG_COS_C[5];
    for (int k = 4; k >= 0; k--) {
        ps = ps * a2 + PG_SIN_C[k];
        pc = pc * a2 + PG_COS_C[k];
    }
    float sa = a + a * (a2 * ps);
    float ca = 1.0f + a2 * pc;
    int qi = (int)q & 3;
    if (qi == 0) { *s_out = sa; *c_out = ca; }
    else if (qi == 1) { *s_out = ca; *c_out = -sa; }
    else if (qi == 2) { *s_out = -sa; *c_out = -ca; }
    else { *s_out = -ca; *c_out = sa; }
}

/* ---------------- value noise ---------------- */
static inline double lattice(int64_t x, int64_t y, int64_t z, uint64_t seed) {
    uint64_t h = seed;
    h = mix64(h ^ (uint64_t)(x * 0x8DA6B343LL));
    h = mix64(h ^ (uint64_t)(y * 0xD8163841LL));
    h = mix64(h ^ (uint64_t)(z * 0xCB1AB31FLL));
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}
static double value_noise(double x, double y, double z, uint64_t seed) {
    double fx = floor(x), fy = floor(y), fz = floor(z);
    int64_t ix = (int64_t)fx, iy = (int64_t)fy, iz = (int64_t)fz;
    double tx = x - fx, ty = y - fy, tz = z - fz;
    double c[2][2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int e = 0; e < 2; e++) c[a][b][e] = lattice(ix + a, iy + b, iz + e, seed);
    double x00 = c[0][0][0] * (1 - tx) + c[1][0][0] * tx;
    double x10 = c[0][1][0] * (1 - tx) + c[1][1][0] * tx;
    double x01 = c[0][0][1] * (1 - tx) + c[1][0][1] * tx;
    double x11 = c[0][1][1] * (1 - tx) + c[1][1][1] * tx;
    double y0 = x00 * (1 - ty) + x10 * ty;
    double y1 = x01 * (1 - ty) + x11 * ty;
    return y0 * (1 - tz) + y1 * tz;
}
static double fbm(const pgrec_config *c, double x, double y, double z) {
    double amp = 1.0, freq = c->fbm_base_freq, sum = 0.0, norm = 0.0;
    for (int o = 0; o < c->fbm_octaves; o++) {
        sum += amp * value_noise(x * freq, y * freq, z * freq, c->seed * 131ULL + (uint64_t)o);
        norm += amp;
        amp *= c->fbm_gain;
        freq *= c->fbm_lacunarity;
    }
    return sum / norm;
}

static void build_medium(pgrec_state *st, const float *albedo_grid) {
    const pgrec_config *c = &st->cfg;
    int64_t G = c->grid_res, nv = G * G * G;
    st->density = (float *)malloc(sizeof(float) * nv);
    st->albedo_grid = (float *)malloc(sizeof(float) * nv);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nv; i++) {
        int64_t ix = i % G, iy = (i / G) % G, iz = i / (G * G);
        double x = (ix + 0.5) / G, y = (iy + 0.5) / G, z = (iz + 0.5) / G;
        double s;
        if (c->medium_kind == 0) {
            s = c->sigma_t_max;
        } else {
            double rx = x - 0.5, ry = y - 0.5, rz = z - 0.5;
            double r = sqrt(rx * rx + ry * ry + rz * rz) / c->cloud_radius;
            double shape = 1.0 - r * r;
            if (shape < 0) shape = 0;
            double v = fbm(c, x, y, z) * shape;
            double t = (v - c->cloud_threshold) / (1.0 - c->cloud_threshold);
            if (t < 0) t = 0;
            t = t * 3.0;
            if (t > 1) t = 1;
            s = c->sigma_t_max * t;
        }
        st->density[i] = (float)s;
        st->albedo_grid[i] = albedo_grid ? albedo_grid[i] : c->albedo;
    }
}

static inline int64_t voxel_of(const pgrec_config *c, float x, float y, float z) {
    int64_t G = c->grid_res;
    float Gf = (float)c->grid_res;
    int64_t ix = (int64_t)floorf(x * Gf), iy = (int64_t)floorf(y * Gf), iz = (int64_t)floorf(z * Gf);
    if (ix < 0) ix = 0;
    if (iy < 0) iy = 0;
    if (iz < 0) iz = 0;
    if (ix >= G) ix = G - 1;
    if (iy >= G) iy = G - 1;
    if (iz >= G) iz = G - 1;
    return ix + G * (iy + G * iz);
}

/* ray / unit-box slab test; returns 0 if missed */
static int box_hit(const float o[3], const float d[3], float *t0, float *t1) {
    float tn = -1e30f, tf = 1e30f;
    for (int a = 0; a < 3; a++) {
        if (fabsf(d[a]) < 1e-30f) {
            if (o[a] < 0.0f || o[a] > 1.0f) return 0;
            continue;
        }
        float inv = 1.0f / d[a];
        float ta = (0.0f - o[a]) * inv, tb = (1.0f - o[a]) * inv;
        if (ta > tb) { float tmp = ta; ta = tb; tb = tmp; }
        if (ta > tn) tn = ta;
        if (tb < tf) tf = tb;
    }
    if (tn > tf) return 0;
    *t0 = tn;
    *t1 = tf;
    return tf > 0.0f;
}

static inline float sigma_t_at(const pgrec_state *st, float x, float y, float z) {
    return st->density[voxel_of(&st->cfg, x, y, z)];
}

/* delta tracking from p along d (p inside or outside the box).
 * Returns 1 and the collision point if a real collision happens. */
static int delta_track(const pgrec_state *st, rng_t *r, const float p[3], const float d[3], float out[3]) {
    float t0, t1;
    float majorant = st->majorant;
    if (majorant <= 0.0f) return 0;
    if (!box_hit(p, d, &t0, &t1)) return 0;
    float inv_maj = 1.0f / majorant;
    float t = t0 > 0.0f ? t0 : 0.0f;
    for (;;) {
        t = t - pg_log(1.0f - rnd(r)) * inv_maj;
        if (t >= t1) return 0;
        float x = p[0] + t * d[0], y = p[1] + t * d[1], z = p[2] + t * d[2];
        float s = sigma_t_at(st, x, y, z);
        if (rnd(r) * majorant < s) {
            out[0] = x; out[1] = y; out[2] = z;
            return 1;
        }
    }
}

/* ratio-tracking transmittance estimate from p along d to the box exit */
static float ratio_track(const pgrec_state *st, rng_t *r, const float p[3], const float d[3]) {
    float t0, t1;
    float majorant = st->majorant;
    if (majorant <= 0.0f) return 1.0f;
    if (!box_hit(p, d, &t0, &t1)) return 1.0f;
    float inv_maj = 1.0f / majorant;
    float t = t0 > 0.0f ? t0 : 0.0f, T = 1.0f;
    for (;;) {
        t = t - pg_log(1.0f - rnd(r)) * inv_maj;
        if (t >= t1) return T;
        float s = sigma_t_at(st, p[0] + t * d[0], p[1] + t * d[1], p[2] + t * d[2]);
        T = T * (1.0f - s * inv_maj);
    }
}

static inline void normalize3(float v[3]) {
    float l = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l; v[1] /= l; v[2] /= l;
}
static inline void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Henyey-Greenstein density for outgoing direction o and light direction d
 * (double: the path tracer's own estimate below) */
static inline double hg_eval(double g, const double o[3], const double d[3]) {
    double od = o[0] * d[0] + o[1] * d[1] + o[2] * d[2];
    double den = 1.0 + g * g + 2.0 * g * od;
    return (1.0 - g * g) / (4.0 * PI_D * den * sqrt(den));
}

/* sample d ~ HG around the travel direction w = -o */
static void hg_sample(float g, const float o[3], rng_t *r, float d[3]) {
    float u1 = rnd(r), u2 = rnd(r), ct;
    if (fabsf(g) < 1e-6f) {
        ct = 1.0f - 2.0f * u1;
    } else {
        float s = (1.0f - g * g) / (1.0f - g + 2.0f * g * u1);
        ct = (1.0f + g * g - s * s) / (2.0f * g);
    }
    if (ct > 1.0f) ct = 1.0f;
    if (ct < -1.0f) ct = -1.0f;
    float st_ = sqrtf(1.0f - ct * ct), sp, cp;
    pg_sincos_2pi(u2, &sp, &cp);
    float w[3] = {-o[0], -o[1], -o[2]}, a[3], u[3], v[3];
    if (fabsf(w[0]) > 0.9f) { a[0] = 0; a[1] = 1; a[2] = 0; } else { a[0] = 1; a[1] = 0; a[2] = 0; }
    cross3(w, a, u); normalize3(u);
    cross3(w, u, v);
    for (int i = 0; i < 3; i++) d[i] = st_ * cp * u[i] + st_ * sp * v[i] + ct * w[i];
    normalize3(d);
}

/* area light: ray from p along d; returns distance to the rectangle or -1 */
static float area_hit(const pgrec_config *c, const float p[3], const float d[3], float *cos_l) {
    float u[3] = {c->area_u[0], c->area_u[1], c->area_u[2]};
    float v[3] = {c->area_v[0], c->area_v[1], c->area_v[2]};
    float n[3];
    cross3(u, v, n);
    normalize3(n);
    float dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    if (dn >= 0.0f) return -1.0f; /* one-sided: visible only from its +n side */
    float q[3] = {c->area_center[0] - p[0], c->area_center[1] - p[1], c->area_center[2] - p[2]};
    float t = (q[0] * n[0] + q[1] * n[1] + q[2] * n[2]) / dn;
    if (t <= 0.0f) return -1.0f;
    float h[3] = {p[0] + t * d[0] - c->area_center[0], p[1] + t * d[1] - c->area_center[1],
                  p[2] + t * d[2] - c->area_center[2]};
    float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    float a = (h[0] * u[0] + h[1] * u[1] + h[2] * u[2]) / uu;
    float b = (h[0] * v[0] + h[1] * v[1] + h[2] * v[2]) / vv;
    if (fabsf(a) > 1.0f || fabsf(b) > 1.0f) return -1.0f;
    *cos_l = -dn;
    return t;
}

static float area_size(const pgrec_config *c) {
    float u[3] = {c->area_u[0], c->area_u[1], c->area_u[2]};
    float v[3] = {c->area_v[0], c->area_v[1], c->area_v[2]}, n[3];
    cross3(u, v, n);
    return 4.0f * sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
}

/* continuous-emitter radiance seen from p along d (ignoring the medium) and
 * the selection-weighted solid-angle pdf of the continuous strategy */
static void continuous_emission(const pgrec_config *c, float p_cont, const float p[3], const float d[3], float *L,
                                float *pdf) {
    int has_area = c->area_radiance > 0, has_sky = c->sky_radiance > 0;
    float pa = has_area ? (has_sky ? c->p_area : 1.0f) : 0.0f;
    float L_ = 0.0f, pdf_ = 0.0f;
    if (has_sky) {
        L_ = L_ + c->sky_radiance;
        pdf_ = pdf_ + (1.0f - pa) * PG_INV_4PI;
    }
    if (has_area) {
        float cl;
        float t = area_hit(c, p, d, &cl);
        if (t > 0) {
            L_ = L_ + c->area_radiance;
            pdf_ = pdf_ + pa * t * t / (area_size(c) * cl);
        }
    }
    *L = L_;
    *pdf = p_cont * pdf_;
}

/* One draw of the emitter-sampling strategy at x: the sun (a delta light)
 * with probability p_sun, else a continuous light (area light or sky, chosen
 * by p_area) sampled by solid angle. Returns the direction toward the light,
 * the radiance it delivers (transmittance to the medium box included; for the
 * sun divided by p_sun) and the continuous strategy's pdf of that direction
 * (selection included; 0 for the sun). */
static void sample_emitter(const pgrec_state *st, rng_t *r, const float x[3], const float sun_to[3], int has_cont,
                           float e[3], float *Le_out, float *pe_out, int *delta_out) {
    const pgrec_config *c = &st->cfg;
    float Le = 0.0f, pe = 0.0f;
    int delta = 0;
    float u = rnd(r);
    if (u < st->p_sun) {
        e[0] = sun_to[0]; e[1] = sun_to[1]; e[2] = sun_to[2];
        delta = 1;
        Le = c->sun_irradiance / st->p_sun * ratio_track(st, r, x, e);
    } else if (has_cont) {
        int has_area = c->area_radiance > 0, has_sky = c->sky_radiance > 0;
        float pa = has_area ? (has_sky ? c->p_area : 1.0f) : 0.0f;
        if (rnd(r) < pa) {
            float a = 2.0f * rnd(r) - 1.0f, bb = 2.0f * rnd(r) - 1.0f, y[3];
            for (int i = 0; i < 3; i++) y[i] = c->area_center[i] + a * c->area_u[i] + bb * c->area_v[i];
            for (int i = 0; i < 3; i++) e[i] = y[i] - x[i];
            normalize3(e);
        } else {
            float z = 1.0f - 2.0f * rnd(r), sp, cp, s = sqrtf(fmaxf(0.0f, 1.0f - z * z));
            pg_sincos_2pi(rnd(r), &sp, &cp);
            e[0] = s * cp; e[1] = s * sp; e[2] = z;
        }
        float Lc, pc;
        continuous_emission(c, 1.0f - st->p_sun, x, e, &Lc, &pc);
        pe = pc;
        /* the lights sit outside the medium box: transmittance to the box exit */
        Le = Lc > 0 ? Lc * ratio_track(st, r, x, e) : 0.0f;
    } else {
        e[0] = sun_to[0]; e[1] = sun_to[1]; e[2] = sun_to[2];
    }
    *Le_out = Le;
    *pe_out = pe;
    *delta_out = delta;
}

static void vbuf_grow(vbuf *b) {
    int64_t nc = b->cap ? b->cap * 2 : 4096;
#define GROW(f, T) b->f = (T *)realloc(b->f, sizeof(T) * nc)
    GROW(px, float); GROW(py, float); GROW(pz, float);
    GROW(ox, float); GROW(oy, float); GROW(oz, float);
    GROW(dx, float); GROW(dy, float); GROW(dz, float);
    GROW(ex, float); GROW(ey, float); GROW(ez, float);
    GROW(g, float); GROW(sigma_s, float); GROW(sigma_t, float); GROW(w_prop, float);
    GROW(Le, float); GROW(pe_e, float); GROW(Lph, float); GROW(pe_ph, float); GROW(L0, float);
    GROW(L0_f64, double);
    GROW(e_delta, uint8_t); GROW(succ_local, int32_t); GROW(voxel, int32_t);
#undef GROW
    b->cap = nc;
}

static inline double f32(double x) { return (double)(float)x; }

/* trace one camera path; appends its vertices to b; returns the path value */
static double trace_path(pgrec_state *st, int64_t pi, vbuf *b, int64_t *first_local, float *bg_out) {
    const pgrec_config *c = &st->cfg;
    rng_t r;
    r.s = mix64(c->seed ^ mix64((uint64_t)pi + 0x632BE59BD9B4E019ULL));
    int64_t pix = pi / c->spp;
    int64_t px_ = pix % c->width, py_ = pix / c->width;
    /* pinhole camera */
    float fwd[3] = {c->cam_target[0] - c->cam_pos[0], c->cam_target[1] - c->cam_pos[1], c->cam_target[2] - c->cam_pos[2]};
    normalize3(fwd);
    float up0[3] = {0, 1, 0}, right[3], up[3];
    cross3(fwd, up0, right); normalize3(right);
    cross3(right, fwd, up);
    float th = st->tan_half_fov;
    float aspect = (float)c->width / (float)c->height;
    float sx = (((float)px_ + rnd(&r)) / (float)c->width * 2.0f - 1.0f) * th * aspect;
    float sy = (1.0f - ((float)py_ + rnd(&r)) / (float)c->height * 2.0f) * th;
    float dir[3];
    for (int i = 0; i < 3; i++) dir[i] = fwd[i] + sx * right[i] + sy * up[i];
    normalize3(dir);
    float pos[3] = {c->cam_pos[0], c->cam_pos[1], c->cam_pos[2]}, x[3];

    *first_local = -1;
    *bg_out = 0.0f;
    const int M = c->extra_direct > 0 ? c->extra_direct : 0;
    for (int i = 0; i < M; i++) { /* paths without a vertex keep empty extra samples */
        int64_t q = pi * M + i;
        st->x_e[3 * q] = 0.0f; st->x_e[3 * q + 1] = 0.0f; st->x_e[3 * q + 2] = 1.0f;
        st->x_Le[q] = 0.0f; st->x_pe[q] = 0.0f; st->x_delta[q] = 0;
    }
    if (!delta_track(st, &r, pos, dir, x)) {
        float L, pdf;
        continuous_emission(c, 1.0f - st->p_sun, pos, dir, &L, &pdf);
        *bg_out = L;
        return (double)L;
    }
    int64_t start = b->n;
    int has_cont = c->sky_radiance > 0 || c->area_radiance > 0;
    float sun_to[3] = {-c->sun_dir[0], -c->sun_dir[1], -c->sun_dir[2]};
    normalize3(sun_to);
    float o[3] = {-dir[0], -dir[1], -dir[2]};
    const float x_first[3] = {x[0], x[1], x[2]};
    for (int depth = 0; depth < c->max_depth; depth++) {
        if (b->n == b->cap) vbuf_grow(b);
        int64_t v = b->n++;
        int64_t vox = voxel_of(c, x[0], x[1], x[2]);
        float sig_t = st->density[vox];
        float alb = st->albedo_grid[vox];
        b->px[v] = x[0]; b->py[v] = x[1]; b->pz[v] = x[2];
        b->ox[v] = o[0]; b->oy[v] = o[1]; b->oz[v] = o[2];
        b->g[v] = c->g;
        b->sigma_t[v] = sig_t;
        b->sigma_s[v] = alb * sig_t;
        b->w_prop[v] = 1.0f / sig_t; /* tau / p_t under delta tracking */
        b->voxel[v] = (int32_t)vox;
        /* emitter sample */
        float e[3], Le, pe;
        int delta;
        sample_emitter(st, &r, x, sun_to, has_cont, e, &Le, &pe, &delta);
        b->ex[v] = e[0]; b->ey[v] = e[1]; b->ez[v] = e[2];
        b->Le[v] = Le;
        b->pe_e[v] = pe;
        b->e_delta[v] = (uint8_t)delta;
        /* phase sample and the continuation */
        float d[3], xn[3];
        hg_sample(c->g, o, &r, d);
        b->dx[v] = d[0]; b->dy[v] = d[1]; b->dz[v] = d[2];
        b->succ_local[v] = -1;
        b->Lph[v] = 0.0f;
        b->pe_ph[v] = 0.0f;
        int hit = delta_track(st, &r, x, d, xn);
        if (!hit) {
            if (has_cont) {
                float Lc, pc;
                continuous_emission(c, 1.0f - st->p_sun, x, d, &Lc, &pc);
                b->Lph[v] = Lc;
                b->pe_ph[v] = pc;
            }
            break;
        }
        if (depth + 1 >= c->max_depth) break; /* truncated: the collision is dropped */
        b->succ_local[v] = (int32_t)(v + 1 - start);
        x[0] = xn[0]; x[1] = xn[1]; x[2] = xn[2];
        o[0] = -d[0]; o[1] = -d[1]; o[2] = -d[2];
    }
    *first_local = start;

    /* extra emitter samples at the first vertex, from a random stream of
     * their own so that the path above is the same with or without them */
    if (M > 0) {
        rng_t rx;
        rx.s = mix64(c->seed ^ mix64((uint64_t)pi + 0xD1B54A32D192ED03ULL) ^ 0x8CB92BA72F3D8DD7ULL);
        for (int i = 0; i < M; i++) {
            float e[3], Le, pe;
            int delta;
            sample_emitter(st, &rx, x_first, sun_to, has_cont, e, &Le, &pe, &delta);
            int64_t q = pi * M + i;
            st->x_e[3 * q] = e[0]; st->x_e[3 * q + 1] = e[1]; st->x_e[3 * q + 2] = e[2];
            st->x_Le[q] = Le;
            st->x_pe[q] = pe;
            st->x_delta[q] = (uint8_t)delta;
        }
    }

    /* Path-tracing estimate from the stored (float32) records, in double:
     * scattered direct radiance per vertex by one-sample balance-heuristic
     * MIS of the emitter and phase samples, then the path throughput. */
    int64_t end = b->n;
    double val = 0.0, beta = f32(b->w_prop[start]);
    for (int64_t v = start; v < end; v++) {
        double ov[3] = {b->ox[v], b->oy[v], b->oz[v]};
        double ev[3] = {b->ex[v], b->ey[v], b->ez[v]};
        double dv[3] = {b->dx[v], b->dy[v], b->dz[v]};
        double gg = b->g[v], ss = b->sigma_s[v];
        double rho_e = hg_eval(gg, ov, ev), rho_d = hg_eval(gg, ov, dv);
        double direct;
        if (b->e_delta[v]) direct = rho_e * (double)b->Le[v];
        else direct = rho_e * (double)b->Le[v] / (rho_e + (double)b->pe_e[v]);
        direct += rho_d * (double)b->Lph[v] / (rho_d + (double)b->pe_ph[v]);
        direct *= ss;
        val += beta * direct;
        if (v + 1 < end) beta *= ss * (double)b->w_prop[v + 1];
        /* store direct temporarily in L0_f64 */
        b->L0_f64[v] = direct;
    }
    /* incoming indirect radiance along d_v: what the rest of the path returns */
    double Lin = 0.0;
    for (int64_t v = end - 1; v >= start; v--) {
        double direct = b->L0_f64[v];
        b->L0_f64[v] = Lin;
        b->L0[v] = (float)Lin;
        if (v > start) Lin = (double)b->w_prop[v] * (direct + (double)b->sigma_s[v] * Lin);
    }
    return val;
}

/* ---------------- public API ---------------- */
void *pgrec_trace(const pgrec_config *cfg, const float *albedo_grid, int32_t nthreads) {
    pgrec_state *st = (pgrec_state *)calloc(1, sizeof(pgrec_state));
    st->cfg = *cfg;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    omp_set_num_threads(nthreads);
#else
    nthreads = 1;
#endif
    build_medium(st, albedo_grid);
    int64_t G = cfg->grid_res, nv = G * G * G;
    float mx = 0.0f;
    for (int64_t i = 0; i < nv; i++) mx = st->density[i] > mx ? st->density[i] : mx;
    st->majorant = mx;
    {
        int has_cont = cfg->sky_radiance > 0 || cfg->area_radiance > 0;
        if (cfg->sun_irradiance <= 0) st->p_sun = 0.0f;
        else if (!has_cont) st->p_sun = 1.0f;
        else st->p_sun = cfg->p_sun;
    }
    st->tan_half_fov = (float)tan(0.5 * cfg->cam_fov_deg * PI_D / 180.0);
    st->n_paths = (int64_t)cfg->width * cfg->height * cfg->spp;
    st->nthreads = nthreads;
    st->bufs = (vbuf *)calloc(nthreads, sizeof(vbuf));
    st->path_first_local = (int64_t *)malloc(sizeof(int64_t) * st->n_paths);
    st->path_thread = (int32_t *)malloc(sizeof(int32_t) * st->n_paths);
    st->bg = (float *)malloc(sizeof(float) * st->n_paths);
    st->val = (double *)malloc(sizeof(double) * st->n_paths);
    if (cfg->extra_direct > 0) {
        int64_t nx = st->n_paths * cfg->extra_direct;
        st->x_e = (float *)malloc(sizeof(float) * 3 * nx);
        st->x_Le = (float *)malloc(sizeof(float) * nx);
        st->x_pe = (float *)malloc(sizeof(float) * nx);
        st->x_delta = (uint8_t *)malloc(nx);
    }
    int64_t np = st->n_paths;
#pragma omp parallel num_threads(nthreads)
    {
        int t = 0, nt = 1;
#ifdef _OPENMP
        t = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        int64_t a = np * t / nt, bnd = np * (t + 1) / nt;
        for (int64_t pi = a; pi < bnd; pi++) {
            st->val[pi] = trace_path(st, pi, &st->bufs[t], &st->path_first_local[pi], &st->bg[pi]);
            st->path_thread[pi] = t;
        }
    }
    st->thread_offset = (int64_t *)malloc(sizeof(int64_t) * (nthreads + 1));
    st->thread_offset[0] = 0;
    for (int t = 0; t < nthreads; t++) st->thread_offset[t + 1] = st->thread_offset[t] + st->bufs[t].n;
    st->n_vertices = st->thread_offset[nthreads];
    return st;
}

int64_t pgrec_num_vertices(void *h) { return ((pgrec_state *)h)->n_vertices; }
int64_t pgrec_num_paths(void *h) { return ((pgrec_state *)h)->n_paths; }
double pgrec_majorant(void *h) { return ((pgrec_state *)h)->majorant; }

/* Copy the records out. Float arrays in the order of `names` below; any
 * pointer may be NULL to skip it. */
void pgrec_copy_vertices(void *h, float **f32_out /* 21 */, double *L0_f64, uint8_t *e_delta, int32_t *succ,
                         int32_t *voxel) {
    pgrec_state *st = (pgrec_state *)h;
#pragma omp parallel for schedule(static, 1)
    for (int t = 0; t < st->nthreads; t++) {
        vbuf *b = &st->bufs[t];
        int64_t off = st->thread_offset[t];
        float *src[21] = {b->px, b->py, b->pz, b->ox, b->oy, b->oz, b->dx, b->dy, b->dz, b->ex, b->ey,
                          b->ez, b->g, b->sigma_s, b->sigma_t, b->w_prop, b->Le, b->pe_e, b->Lph, b->pe_ph, b->L0};
        for (int f = 0; f < 21; f++)
            if (f32_out[f]) memcpy(f32_out[f] + off, src[f], sizeof(float) * b->n);
        if (L0_f64) memcpy(L0_f64 + off, b->L0_f64, sizeof(double) * b->n);
        if (e_delta) memcpy(e_delta + off, b->e_delta, b->n);
        if (voxel) memcpy(voxel + off, b->voxel, sizeof(int32_t) * b->n);
        if (succ) {
            /* succ_local is an offset within the path; each vertex's path start is
             * recovered by walking: vertex v has succ v+1 inside the same buffer */
            for (int64_t v = 0; v < b->n; v++)
                succ[off + v] = b->succ_local[v] < 0 ? -1 : (int32_t)(off + v + 1);
        }
    }
}

void pgrec_copy_paths(void *h, int32_t *first, float *bg, double *val) {
    pgrec_state *st = (pgrec_state *)h;
#pragma omp parallel for schedule(static)
    for (int64_t pi = 0; pi < st->n_paths; pi++) {
        int64_t fl = st->path_first_local[pi];
        if (first) first[pi] = fl < 0 ? -1 : (int32_t)(st->thread_offset[st->path_thread[pi]] + fl);
        if (bg) bg[pi] = st->bg[pi];
        if (val) val[pi] = st->val[pi];
    }
}

/* Extra emitter samples at the first vertices (extra_direct per path, path
 * p's at [p * extra_direct, (p + 1) * extra_direct)); directions split into
 * x, y, z arrays. */
void pgrec_copy_extra(void *h, float *ex, float *ey, float *ez, float *Le, float *pe, uint8_t *delta) {
    pgrec_state *st = (pgrec_state *)h;
    int64_t nx = st->n_paths * (st->cfg.extra_direct > 0 ? st->cfg.extra_direct : 0);
    for (int64_t q = 0; q < nx; q++) {
        ex[q] = st->x_e[3 * q];
        ey[q] = st->x_e[3 * q + 1];
        ez[q] = st->x_e[3 * q + 2];
        Le[q] = st->x_Le[q];
        pe[q] = st->x_pe[q];
        delta[q] = st->x_delta[q];
    }
}

void pgrec_copy_medium(void *h, float *density, float *albedo) {
    pgrec_state *st = (pgrec_state *)h;
    int64_t G = st->cfg.grid_res, nv = G * G * G;
    if (density) memcpy(density, st->density, sizeof(float) * nv);
    if (albedo) memcpy(albedo, st->albedo_grid, sizeof(float) * nv);
}

void pgrec_free(void *h) {
    pgrec_state *st = (pgrec_state *)h;
    if (!st) return;
    for (int t = 0; t < st->nthreads; t++) {
        vbuf *b = &st->bufs[t];
        void *ptrs[] = {b->px, b->py, b->pz, b->ox, b->oy, b->oz, b->dx, b->dy, b->dz, b->ex, b->ey, b->ez,
                        b->g, b->sigma_s, b->sigma_t, b->w_prop, b->Le, b->pe_e, b->Lph, b->pe_ph, b->L0,
                        b->L0_f64, b->e_delta, b->succ_local, b->voxel};
        for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
    }
    free(st->bufs);
    free(st->path_first_local);
    free(st->path_thread);
    free(st->bg);
    free(st->val);
    free(st->x_e);
    free(st->x_Le);
    free(st->x_pe);
    free(st->x_delta);
    free(st->thread_offset);
    free(st->density);
    free(st->albedo_grid);
    free(st);
}

/* the medium grids alone (grid_res^3 sigma_t and albedo), as pgrec_trace builds them */
void pgrec_build_medium(const pgrec_config *cfg, const float *albedo_grid, float *density_out, float *albedo_out) {
    pgrec_state st;
    memset(&st, 0, sizeof(st));
    st.cfg = *cfg;
    build_medium(&st, albedo_grid);
    int64_t G = cfg->grid_res, nv = G * G * G;
    memcpy(density_out, st.density, sizeof(float) * nv);
    memcpy(albedo_out, st.albedo_grid, sizeof(float) * nv);
    free(st.density);
    free(st.albedo_grid);
}

/* the recorder's elementary functions, exported for their tests */
float pgrec_log(float x) { return pg_log(x); }
void pgrec_sincos_2pi(float u, float *s, float *c) { pg_sincos_2pi(u, s, c); }
