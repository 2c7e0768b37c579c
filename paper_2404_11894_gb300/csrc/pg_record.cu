// GPU path recorder: the instrumented volumetric path tracer of Section 4
// ("Instrumented path tracer": per shading point the emitter-sampling and
// phase-sampling records and the incoming indirect radiance, a path's points
// stored contiguously in path order) run on the device, one thread per path.
//
// Delta tracking through a piecewise-constant voxel medium, emitter samples
// with ratio-tracking transmittance and exact Henyey-Greenstein sampling in
// single precision (this GPU's double-precision rate is a small fraction of
// its single-precision one); the path tracer's own balance-heuristic
// estimate, from the stored float records, in double. The arithmetic is the
// host recorder's, operation for operation: only IEEE-rounded +, -, *, /,
// sqrt and exact operations (frexp, floor, integer hashing), the logarithm
// and sin/cos of 2 pi u by their own series. This file is compiled without
// FMA contraction, so the device and the host recorder produce bit-identical
// records from the same scene and seed.
//
// Two passes over the same random streams: the first counts each path's
// vertices (their exclusive scan gives every path its slice of the output,
// in path order), the second writes the records.
#include <math.h>

#include "pg_internal.cuh"

namespace {

constexpr double PI_D = 3.14159265358979323846;
constexpr float INV_4PI_F = 0.07957746833562851f;

struct Scn {
    pg_scene c;         // the caller's scene (floats, as given)
    float p_sun;        // probability that an emitter sample picks the sun
    float th;           // tan(fov/2), from the host C library as the host recorder takes it
};

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// uniform on [0, 1) with 24 random bits (exact in float)
__device__ __forceinline__ float rnd(uint64_t &s) {
    s += 0x9E3779B97F4A7C15ULL;
    return (float)(mix64(s) >> 40) * (1.0f / 16777216.0f);
}

// log x: x = m 2^e, m in [1/sqrt2, sqrt2), log m = 2 artanh((m-1)/(m+1)) by
// its odd series to the 11th power, ln2 split into a 12-bit head and a tail
__device__ float rec_log(float x) {
    int e;
    float m = frexpf(x, &e);
    if (m < 0.7071067690849304f) {
        m = m * 2.0f;
        e = e - 1;
    }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    float p = 0.09090909361839294f;
    p = p * s2 + 0.1111111119389534f;
    p = p * s2 + 0.1428571492433548f;
    p = p * s2 + 0.20000000298023224f;
    p = p * s2 + 0.3333333432674408f;
    p = p * s2 + 1.0f;
    const float lm = 2.0f * s * p;
    return (float)e * 0.693115234375f + ((float)e * 3.194618329871446e-05f + lm);
}

// sin and cos of 2 pi u, u in [0, 1): quadrant by 4u = q + f, Taylor series
// of sin and cos on [0, pi/2) to the 13th / 12th power
__device__ void rec_sincos_2pi(float u, float &so, float &co) {
    const float t = 4.0f * u;
    const float q = floorf(t);
    const float f = t - q;
    const float a = f * 1.5707963705062866f;
    const float a2 = a * a;
    float ps = 1.6059044372074283e-10f, pc = 2.0876755879584152e-09f;
    ps = ps * a2 + -2.5052107943679403e-08f;
    pc = pc * a2 + -2.755731998149713e-07f;
    ps = ps * a2 + 2.7557318844628753e-06f;
    pc = pc * a2 + 2.4801587642286904e-05f;
    ps = ps * a2 + -0.00019841270113829523f;
    pc = pc * a2 + -0.0013888889225199819f;
    ps = ps * a2 + 0.008333333767950535f;
    pc = pc * a2 + 0.0416666679084301f;
    ps = ps * a2 + -0.1666666716337204f;
    pc = pc * a2 + -0.5f;
    const float sa = a + a * (a2 * ps);
    const float ca = 1.0f + a2 * pc;
    const int qi = (int)q & 3;
    if (qi == 0) { so = sa; co = ca; }
    else if (qi == 1) { so = ca; co = -sa; }
    else if (qi == 2) { so = -sa; co = -ca; }
    else { so = -ca; co = sa; }
}

__device__ __forceinline__ void normalize3(float v[3]) {
    const float l = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] = v[0] / l;
    v[1] = v[1] / l;
    v[2] = v[2] / l;
}
__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ int64_t voxel_of(const pg_scene &c, float x, float y, float z) {
    const int64_t G = c.grid_res;
    const float Gf = (float)c.grid_res;
    int64_t ix = (int64_t)floorf(x * Gf), iy = (int64_t)floorf(y * Gf), iz = (int64_t)floorf(z * Gf);
    ix = ix < 0 ? 0 : (ix >= G ? G - 1 : ix);
    iy = iy < 0 ? 0 : (iy >= G ? G - 1 : iy);
    iz = iz < 0 ? 0 : (iz >= G ? G - 1 : iz);
    return ix + G * (iy + G * iz);
}

// ray against the unit box [0,1]^3: entry and exit distances, 0 if missed
__device__ int box_hit(const float o[3], const float d[3], float &t0, float &t1) {
    float tn = -1e30f, tf = 1e30f;
    for (int a = 0; a < 3; a++) {
        if (fabsf(d[a]) < 1e-30f) {
            if (o[a] < 0.0f || o[a] > 1.0f) return 0;
            continue;
        }
        const float inv = 1.0f / d[a];
        float ta = (0.0f - o[a]) * inv, tb = (1.0f - o[a]) * inv;
        if (ta > tb) {
            const float tmp = ta;
            ta = tb;
            tb = tmp;
        }
        if (ta > tn) tn = ta;
        if (tb < tf) tf = tb;
    }
    if (tn > tf) return 0;
    t0 = tn;
    t1 = tf;
    return tf > 0.0f;
}

// delta tracking from p along d: 1 and the collision point, or 0 (left the box)
__device__ int delta_track(const Scn &S, const float *__restrict__ dens, float maj, uint64_t &r, const float p[3],
                           const float d[3], float out[3]) {
    float t0, t1;
    if (maj <= 0.0f) return 0;
    if (!box_hit(p, d, t0, t1)) return 0;
    const float inv_maj = 1.0f / maj;
    float t = t0 > 0.0f ? t0 : 0.0f;
    for (;;) {
        t = t - rec_log(1.0f - rnd(r)) * inv_maj;
        if (t >= t1) return 0;
        const float x = p[0] + t * d[0], y = p[1] + t * d[1], z = p[2] + t * d[2];
        const float s = __ldg(dens + voxel_of(S.c, x, y, z));
        if (rnd(r) * maj < s) {
            out[0] = x;
            out[1] = y;
            out[2] = z;
            return 1;
        }
    }
}

// ratio-tracking transmittance from p along d to the box exit
__device__ float ratio_track(const Scn &S, const float *__restrict__ dens, float maj, uint64_t &r, const float p[3],
                             const float d[3]) {
    float t0, t1;
    if (maj <= 0.0f) return 1.0f;
    if (!box_hit(p, d, t0, t1)) return 1.0f;
    const float inv_maj = 1.0f / maj;
    float t = t0 > 0.0f ? t0 : 0.0f, T = 1.0f;
    for (;;) {
        t = t - rec_log(1.0f - rnd(r)) * inv_maj;
        if (t >= t1) return T;
        const float s = __ldg(dens + voxel_of(S.c, p[0] + t * d[0], p[1] + t * d[1], p[2] + t * d[2]));
        T = T * (1.0f - s * inv_maj);
    }
}

// Henyey-Greenstein density in double (the path tracer's own estimate)
__device__ __forceinline__ double hg_eval(double g, const double o[3], const double d[3]) {
    const double od = o[0] * d[0] + o[1] * d[1] + o[2] * d[2];
    const double den = 1.0 + g * g + 2.0 * g * od;
    return (1.0 - g * g) / (4.0 * PI_D * den * sqrt(den));
}

// d ~ HG around the travel direction w = -o
__device__ void hg_sample(float g, const float o[3], uint64_t &r, float d[3]) {
    const float u1 = rnd(r), u2 = rnd(r);
    float ct;
    if (fabsf(g) < 1e-6f) {
        ct = 1.0f - 2.0f * u1;
    } else {
        const float s = (1.0f - g * g) / (1.0f - g + 2.0f * g * u1);
        ct = (1.0f + g * g - s * s) / (2.0f * g);
    }
    if (ct > 1.0f) ct = 1.0f;
    if (ct < -1.0f) ct = -1.0f;
    const float st = sqrtf(1.0f - ct * ct);
    float sp, cp;
    rec_sincos_2pi(u2, sp, cp);
    float w[3] = {-o[0], -o[1], -o[2]}, a[3], u[3], v[3];
    if (fabsf(w[0]) > 0.9f) {
        a[0] = 0; a[1] = 1; a[2] = 0;
    } else {
        a[0] = 1; a[1] = 0; a[2] = 0;
    }
    cross3(w, a, u);
    normalize3(u);
    cross3(w, u, v);
    for (int i = 0; i < 3; i++) d[i] = st * cp * u[i] + st * sp * v[i] + ct * w[i];
    normalize3(d);
}

// one-sided rectangular light: distance along d from p, or -1
__device__ float area_hit(const pg_scene &c, const float p[3], const float d[3], float &cos_l) {
    float u[3] = {c.area_u[0], c.area_u[1], c.area_u[2]};
    float v[3] = {c.area_v[0], c.area_v[1], c.area_v[2]};
    float n[3];
    cross3(u, v, n);
    normalize3(n);
    const float dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    if (dn >= 0.0f) return -1.0f;
    const float q[3] = {c.area_center[0] - p[0], c.area_center[1] - p[1], c.area_center[2] - p[2]};
    const float t = (q[0] * n[0] + q[1] * n[1] + q[2] * n[2]) / dn;
    if (t <= 0.0f) return -1.0f;
    const float h[3] = {p[0] + t * d[0] - c.area_center[0], p[1] + t * d[1] - c.area_center[1],
                        p[2] + t * d[2] - c.area_center[2]};
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const float a = (h[0] * u[0] + h[1] * u[1] + h[2] * u[2]) / uu;
    const float b = (h[0] * v[0] + h[1] * v[1] + h[2] * v[2]) / vv;
    if (fabsf(a) > 1.0f || fabsf(b) > 1.0f) return -1.0f;
    cos_l = -dn;
    return t;
}

__device__ float area_size(const pg_scene &c) {
    float u[3] = {c.area_u[0], c.area_u[1], c.area_u[2]};
    float v[3] = {c.area_v[0], c.area_v[1], c.area_v[2]}, n[3];
    cross3(u, v, n);
    return 4.0f * sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
}

// continuous-light radiance along d from p (medium ignored) and the
// continuous strategy's solid-angle pdf, selection p_cont included
__device__ void continuous_emission(const pg_scene &c, float p_cont, const float p[3], const float d[3], float &L,
                                    float &pdf) {
    const int has_area = c.area_radiance > 0, has_sky = c.sky_radiance > 0;
    const float pa = has_area ? (has_sky ? c.p_area : 1.0f) : 0.0f;
    float L_ = 0.0f, pdf_ = 0.0f;
    if (has_sky) {
        L_ = L_ + c.sky_radiance;
        pdf_ = pdf_ + (1.0f - pa) * INV_4PI_F;
    }
    if (has_area) {
        float cl;
        const float t = area_hit(c, p, d, cl);
        if (t > 0) {
            L_ = L_ + c.area_radiance;
            pdf_ = pdf_ + pa * t * t / (area_size(c) * cl);
        }
    }
    L = L_;
    pdf = p_cont * pdf_;
}

// one draw of the emitter strategy at x (sun with probability p_sun, else a
// continuous light by solid angle), with ratio-tracking transmittance
__device__ void sample_emitter(const Scn &S, const float *__restrict__ dens, float maj, uint64_t &r,
                               const float x[3], const float sun_to[3], int has_cont, float e[3], float &Le_out,
                               float &pe_out, int &delta_out) {
    const pg_scene &c = S.c;
    float Le = 0.0f, pe = 0.0f;
    int delta = 0;
    const float u = rnd(r);
    if (u < S.p_sun) {
        e[0] = sun_to[0]; e[1] = sun_to[1]; e[2] = sun_to[2];
        delta = 1;
        Le = c.sun_irradiance / S.p_sun * ratio_track(S, dens, maj, r, x, e);
    } else if (has_cont) {
        const int has_area = c.area_radiance > 0, has_sky = c.sky_radiance > 0;
        const float pa = has_area ? (has_sky ? c.p_area : 1.0f) : 0.0f;
        if (rnd(r) < pa) {
            const float a = 2.0f * rnd(r) - 1.0f, bb = 2.0f * rnd(r) - 1.0f;
            float y[3];
            for (int i = 0; i < 3; i++) y[i] = c.area_center[i] + a * c.area_u[i] + bb * c.area_v[i];
            for (int i = 0; i < 3; i++) e[i] = y[i] - x[i];
            normalize3(e);
        } else {
            const float z = 1.0f - 2.0f * rnd(r);
            float sp, cp;
            const float s = sqrtf(fmaxf(0.0f, 1.0f - z * z));
            rec_sincos_2pi(rnd(r), sp, cp);
            e[0] = s * cp; e[1] = s * sp; e[2] = z;
        }
        float Lc, pc;
        continuous_emission(c, 1.0f - S.p_sun, x, e, Lc, pc);
        pe = pc;
        Le = Lc > 0 ? Lc * ratio_track(S, dens, maj, r, x, e) : 0.0f;
    } else {
        e[0] = sun_to[0]; e[1] = sun_to[1]; e[2] = sun_to[2];
    }
    Le_out = Le;
    pe_out = pe;
    delta_out = delta;
}

__device__ __forceinline__ double f32(double x) { return (double)(float)x; }

// One camera path per thread. WRITE = false: count its vertices into cnt[p].
// WRITE = true: write them at off[p].. and the path's outputs.
template <bool WRITE>
__global__ void __launch_bounds__(128) record_kernel(Scn S, const float *__restrict__ dens,
                                                     const float *__restrict__ alb, const float *__restrict__ d_maj,
                                                     int64_t n_paths, int64_t *__restrict__ cnt,
                                                     const int64_t *__restrict__ off, pg_recording out) {
    const int64_t pi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= n_paths) return;
    const pg_scene &c = S.c;
    const float maj = *d_maj;
    uint64_t r = mix64(c.seed ^ mix64((uint64_t)pi + 0x632BE59BD9B4E019ULL));
    const int64_t pix = pi / c.spp;
    const int64_t px_ = pix % c.width, py_ = pix / c.width;
    float fwd[3] = {c.cam_target[0] - c.cam_pos[0], c.cam_target[1] - c.cam_pos[1], c.cam_target[2] - c.cam_pos[2]};
    normalize3(fwd);
    float up0[3] = {0, 1, 0}, right[3], up[3];
    cross3(fwd, up0, right);
    normalize3(right);
    cross3(right, fwd, up);
    const float aspect = (float)c.width / (float)c.height;
    const float sx = (((float)px_ + rnd(r)) / (float)c.width * 2.0f - 1.0f) * S.th * aspect;
    const float sy = (1.0f - ((float)py_ + rnd(r)) / (float)c.height * 2.0f) * S.th;
    float dir[3];
    for (int i = 0; i < 3; i++) dir[i] = fwd[i] + sx * right[i] + sy * up[i];
    normalize3(dir);
    const float pos[3] = {c.cam_pos[0], c.cam_pos[1], c.cam_pos[2]};
    float x[3];
    const int M = c.extra_direct > 0 ? c.extra_direct : 0;
    if (WRITE) {
        for (int i = 0; i < M; i++) {
            const int64_t q = pi * M + i;
            out.x_ex[q] = 0.0f; out.x_ey[q] = 0.0f; out.x_ez[q] = 1.0f;
            out.x_Le[q] = 0.0f; out.x_pe[q] = 0.0f; out.x_delta[q] = 0;
        }
    }
    if (!delta_track(S, dens, maj, r, pos, dir, x)) {
        if (WRITE) {
            float L, pdf;
            continuous_emission(c, 1.0f - S.p_sun, pos, dir, L, pdf);
            out.first[pi] = -1;
            out.bg[pi] = L;
            if (out.val) out.val[pi] = (double)L;
        } else {
            cnt[pi] = 0;
        }
        return;
    }
    const int64_t start = WRITE ? off[pi] : 0;
    const int has_cont = c.sky_radiance > 0 || c.area_radiance > 0;
    float sun_to[3] = {-c.sun_dir[0], -c.sun_dir[1], -c.sun_dir[2]};
    normalize3(sun_to);
    float o[3] = {-dir[0], -dir[1], -dir[2]};
    const float x_first[3] = {x[0], x[1], x[2]};
    int64_t nv = 0;
    for (int depth = 0; depth < c.max_depth; depth++) {
        const int64_t v = start + nv++;
        const int64_t vox = voxel_of(c, x[0], x[1], x[2]);
        const float sig_t = __ldg(dens + vox);
        const float al = __ldg(alb + vox);
        if (WRITE) {
            out.px[v] = x[0]; out.py[v] = x[1]; out.pz[v] = x[2];
            out.ox[v] = o[0]; out.oy[v] = o[1]; out.oz[v] = o[2];
            out.g[v] = c.g;
            out.sigma_t[v] = sig_t;
            out.sigma_s[v] = al * sig_t;
            out.w_prop[v] = 1.0f / sig_t;
            if (out.voxel) out.voxel[v] = (int32_t)vox;
        }
        float e[3], Le, pe;
        int delta;
        sample_emitter(S, dens, maj, r, x, sun_to, has_cont, e, Le, pe, delta);
        float d[3], xn[3];
        hg_sample(c.g, o, r, d);
        if (WRITE) {
            out.ex[v] = e[0]; out.ey[v] = e[1]; out.ez[v] = e[2];
            out.Le[v] = Le;
            out.pe_e[v] = pe;
            out.e_delta[v] = (uint8_t)delta;
            out.dx[v] = d[0]; out.dy[v] = d[1]; out.dz[v] = d[2];
            out.succ[v] = -1;
            out.Lph[v] = 0.0f;
            out.pe_ph[v] = 0.0f;
        }
        const int hit = delta_track(S, dens, maj, r, x, d, xn);
        if (!hit) {
            if (WRITE && has_cont) {
                float Lc, pc;
                continuous_emission(c, 1.0f - S.p_sun, x, d, Lc, pc);
                out.Lph[v] = Lc;
                out.pe_ph[v] = pc;
            }
            break;
        }
        if (depth + 1 >= c.max_depth) break; // truncated: the collision is dropped
        if (WRITE) out.succ[v] = (int32_t)(v + 1);
        x[0] = xn[0]; x[1] = xn[1]; x[2] = xn[2];
        o[0] = -d[0]; o[1] = -d[1]; o[2] = -d[2];
    }
    if (!WRITE) {
        cnt[pi] = nv;
        return;
    }
    out.first[pi] = (int32_t)start;
    out.bg[pi] = 0.0f;

    // extra emitter samples at the first vertex, on a random stream of their own
    if (M > 0) {
        uint64_t rx = mix64(c.seed ^ mix64((uint64_t)pi + 0xD1B54A32D192ED03ULL) ^ 0x8CB92BA72F3D8DD7ULL);
        for (int i = 0; i < M; i++) {
            float e[3], Le, pe;
            int delta;
            sample_emitter(S, dens, maj, rx, x_first, sun_to, has_cont, e, Le, pe, delta);
            const int64_t q = pi * M + i;
            out.x_ex[q] = e[0]; out.x_ey[q] = e[1]; out.x_ez[q] = e[2];
            out.x_Le[q] = Le;
            out.x_pe[q] = pe;
            out.x_delta[q] = (uint8_t)delta;
        }
    }

    // the path tracer's own estimate from the stored float records: per
    // vertex the one-sample balance-heuristic direct light, the throughput
    // along the path, then the incoming indirect radiance from the end back
    const int64_t end = start + nv;
    double val = 0.0, beta = f32(out.w_prop[start]);
    for (int64_t v = start; v < end; v++) {
        const double ov[3] = {out.ox[v], out.oy[v], out.oz[v]};
        const double ev[3] = {out.ex[v], out.ey[v], out.ez[v]};
        const double dv[3] = {out.dx[v], out.dy[v], out.dz[v]};
        const double gg = out.g[v], ss = out.sigma_s[v];
        const double rho_e = hg_eval(gg, ov, ev), rho_d = hg_eval(gg, ov, dv);
        double direct;
        if (out.e_delta[v]) direct = rho_e * (double)out.Le[v];
        else direct = rho_e * (double)out.Le[v] / (rho_e + (double)out.pe_e[v]);
        direct += rho_d * (double)out.Lph[v] / (rho_d + (double)out.pe_ph[v]);
        direct *= ss;
        val += beta * direct;
        if (v + 1 < end) beta *= ss * (double)out.w_prop[v + 1];
        out.L0_f64[v] = direct;
    }
    double Lin = 0.0;
    for (int64_t v = end - 1; v >= start; v--) {
        const double direct = out.L0_f64[v];
        out.L0_f64[v] = Lin;
        out.L0[v] = (float)Lin;
        if (v > start) Lin = (double)out.w_prop[v] * (direct + (double)out.sigma_s[v] * Lin);
    }
    if (out.val) out.val[pi] = val;
}

// majorant = max sigma_t over the grid: non-negative floats order like their bits
__global__ void grid_max_kernel(const float *__restrict__ dens, int64_t nv, float *__restrict__ mx,
                                int32_t *__restrict__ flags) {
    float m = 0.0f;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const float s = dens[i];
        if (!isfinite(s) || s < 0.0f) bad = 1;
        else m = fmaxf(m, s);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<int *>(mx), __float_as_int(m));
        if (bad) atomicOr(flags, PG_FLAG_BAD_RANGE);
    }
}

__global__ void albedo_check_kernel(const float *__restrict__ alb, int64_t nv, int32_t *__restrict__ flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = alb[i];
        if (!isfinite(a) || a < 0.0f) atomicOr(flags, PG_FLAG_BAD_RANGE);
    }
}

pg_status check_scene(const pg_scene *sc, Scn &S) {
    if (!sc) return PG_ERR_INVALID_ARG;
    const pg_scene &c = *sc;
    if (c.grid_res < 1 || c.grid_res > 2048 || !c.density || !c.albedo) return PG_ERR_INVALID_ARG;
    if (c.width < 1 || c.height < 1 || c.spp < 1 || c.max_depth < 1 || c.extra_direct < 0) return PG_ERR_INVALID_ARG;
    if (!(fabsf(c.g) < 1.0f)) return PG_ERR_INVALID_ARG;
    if (!(c.sun_irradiance >= 0.0f) || !(c.sky_radiance >= 0.0f) || !(c.area_radiance >= 0.0f))
        return PG_ERR_INVALID_ARG;
    if (!(c.cam_fov_deg > 0.0f && c.cam_fov_deg < 180.0f)) return PG_ERR_INVALID_ARG;
    const int64_t n_paths = (int64_t)c.width * c.height * c.spp;
    if (n_paths >= INT32_MAX) return PG_ERR_INVALID_ARG;
    S.c = c;
    const int has_cont = c.sky_radiance > 0 || c.area_radiance > 0;
    if (c.sun_irradiance <= 0) S.p_sun = 0.0f;
    else if (!has_cont) S.p_sun = 1.0f;
    else S.p_sun = c.p_sun;
    if (c.sun_irradiance > 0 && has_cont && !(c.p_sun > 0.0f && c.p_sun < 1.0f)) return PG_ERR_INVALID_ARG;
    // host math library, as the host recorder evaluates it
    S.th = (float)tan(0.5 * c.cam_fov_deg * PI_D / 180.0);
    return PG_OK;
}

// the majorant into d_mx (device), validating the grids
pg_status majorant(const pg_scene &c, float *d_mx, int32_t *flags, cudaStream_t s) {
    const int64_t nv = (int64_t)c.grid_res * c.grid_res * c.grid_res;
    PG_CUDA(cudaMemsetAsync(d_mx, 0, 4, s));
    PG_CUDA(cudaMemsetAsync(flags, 0, 4, s));
    const int blocks = (int)std::min<int64_t>((nv + 255) / 256, (int64_t)pg_num_sms() * 8);
    grid_max_kernel<<<blocks, 256, 0, s>>>(c.density, nv, d_mx, flags);
    albedo_check_kernel<<<blocks, 256, 0, s>>>(c.albedo, nv, flags);
    pg_count_launches(2);
    PG_LAUNCH_CHECK();
    return PG_OK;
}

} // namespace

extern "C" pg_status pg_record_count(const pg_scene *scene, int64_t *path_offsets, int64_t *n_vertices,
                                     pg_stream_t stream) {
    Scn S;
    PG_TRY(check_scene(scene, S));
    if (!path_offsets || !n_vertices) return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_paths = (int64_t)S.c.width * S.c.height * S.c.spp;
    float *mx = nullptr;
    PG_TRY(pg_alloc(nullptr, (void **)&mx, 16, s));
    int32_t *flags = reinterpret_cast<int32_t *>(mx) + 1;
    pg_status st = majorant(S.c, mx, flags, s);
    pg_recording none = {};
    if (st == PG_OK) {
        record_kernel<false><<<pg_blocks(n_paths, 128), 128, 0, s>>>(S, S.c.density, S.c.albedo, mx, n_paths,
                                                                    path_offsets, nullptr, none);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    int64_t total = 0;
    if (st == PG_OK) st = pg_scan_exclusive64(nullptr, path_offsets, n_paths + 1, nullptr, s);
    int32_t hflags = 0;
    if (st == PG_OK && (cudaMemcpyAsync(&total, path_offsets + n_paths, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaMemcpyAsync(&hflags, flags, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = PG_ERR_CUDA;
    cudaFreeAsync(mx, s);
    if (st != PG_OK) {
        (void)cudaGetLastError();
        return st;
    }
    if (hflags) return PG_ERR_INVALID_ARG;
    if (total >= INT32_MAX) return PG_ERR_UNSUPPORTED;
    *n_vertices = total;
    return PG_OK;
}

extern "C" pg_status pg_record_fill(const pg_scene *scene, const int64_t *path_offsets, const pg_recording *out,
                                    pg_stream_t stream) {
    Scn S;
    PG_TRY(check_scene(scene, S));
    if (!path_offsets || !out) return PG_ERR_INVALID_ARG;
    const pg_recording &o = *out;
    if (!o.px || !o.py || !o.pz || !o.ox || !o.oy || !o.oz || !o.dx || !o.dy || !o.dz || !o.ex || !o.ey || !o.ez ||
        !o.g || !o.sigma_s || !o.sigma_t || !o.w_prop || !o.Le || !o.pe_e || !o.Lph || !o.pe_ph || !o.L0 ||
        !o.L0_f64 || !o.e_delta || !o.succ || !o.first || !o.bg)
        return PG_ERR_INVALID_ARG;
    if (S.c.extra_direct > 0 && (!o.x_ex || !o.x_ey || !o.x_ez || !o.x_Le || !o.x_pe || !o.x_delta))
        return PG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_paths = (int64_t)S.c.width * S.c.height * S.c.spp;
    float *mx = nullptr;
    PG_TRY(pg_alloc(nullptr, (void **)&mx, 16, s));
    int32_t *flags = reinterpret_cast<int32_t *>(mx) + 1;
    pg_status st = majorant(S.c, mx, flags, s);
    if (st == PG_OK) {
        record_kernel<true><<<pg_blocks(n_paths, 128), 128, 0, s>>>(S, S.c.density, S.c.albedo, mx, n_paths,
                                                                   nullptr, path_offsets, o);
        pg_count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = PG_ERR_CUDA;
    }
    cudaFreeAsync(mx, s);
    return st;
}
