/*
 * synth_site.c -- ray caster of the merged multi-station site scan.
 *
 * INPUT GENERATOR ONLY: it holds none of the decimation arithmetic.  It
 * produces the massive merged clouds (up to a billion points) that both the
 * CUDA path and the CPU oracle consume; synth.py places the scene's
 * primitives and the stations with numpy's PCG64 and hands them here.
 *
 * Scene: the inside of the closed box [0,W] x [0,D] x [0,H] (ground, four
 * walls, roof) with axis-aligned boxes standing on the ground and vertical
 * cylinders.  Every station casts n_az x n_el rays on a regular azimuth x
 * elevation grid (elevation from -90 to +90 degrees, so the density peaks at
 * the poles of each station, as with a stationary terrestrial scanner).  The
 * site is closed, so every ray returns: station s, ray i = az * n_el + el is
 * written to row s * n_az * n_el + i.  Range noise is Gaussian with standard
 * deviation sigma metres; its two uniforms per ray come from splitmix64
 * (Steele, Lea, Flood, OOPSLA 2014) of (seed, station, ray), turned into a
 * normal deviate by the Box-Muller transform, so the output does not depend
 * on the thread count.  Hits are quantised with floor(1000 x + 0.5) to int32
 * millimetres; colour is the object's colour times a 0.5 m checker (1.0 or
 * 0.6).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t splitmix64(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* uniform in (0, 1]: 53 random bits */
static inline double unit53(uint64_t x) { return ((double)(x >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

typedef struct {
    int kind; /* 0 box from outside, 1 vertical cylinder */
    double lo[3], hi[3];  /* box */
    double cx, cy, r, h;  /* cylinder */
    double bcx, bcy, br;  /* bounding circle in the xy plane */
    double rgb[3];
} prim_t;

/* exit distance from inside the site box */
static inline double box_exit(const double o[3], const double d[3], const double size[3],
                              int* axis) {
    double best = INFINITY;
    int ax = 0;
    for (int a = 0; a < 3; a++) {
        double t;
        if (d[a] > 0) t = (size[a] - o[a]) / d[a];
        else if (d[a] < 0) t = (0.0 - o[a]) / d[a];
        else continue;
        if (t < best) {
            best = t;
            ax = a;
        }
    }
    *axis = ax;
    return best;
}

static inline double box_enter(const double o[3], const double d[3], const double lo[3],
                               const double hi[3]) {
    double tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; a++) {
        if (d[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi[a]) return INFINITY;
            continue;
        }
        double t1 = (lo[a] - o[a]) / d[a], t2 = (hi[a] - o[a]) / d[a];
        double a1 = t1 < t2 ? t1 : t2, a2 = t1 < t2 ? t2 : t1;
        if (a1 > tn) tn = a1;
        if (a2 < tf) tf = a2;
    }
    if (tn <= tf && tn > 1e-9) return tn;
    return INFINITY;
}

static inline double cyl_enter(const double o[3], const double d[3], const prim_t* p) {
    double ox = o[0] - p->cx, oy = o[1] - p->cy;
    double a = d[0] * d[0] + d[1] * d[1];
    if (a <= 0.0) return INFINITY;
    double b = ox * d[0] + oy * d[1];
    double c = ox * ox + oy * oy - p->r * p->r;
    double disc = b * b - a * c;
    if (disc < 0) return INFINITY;
    double t = (-b - sqrt(disc)) / a;
    if (!(t > 1e-9)) return INFINITY;
    double z = o[2] + t * d[2];
    if (z < 0.0 || z > p->h) return INFINITY;
    return t;
}

/*
 * prims: nprim records of 17 doubles each:
 *   kind, lo[3], hi[3], cx, cy, r, h, bcx, bcy, br, rgb[3]
 * stations: nst x 3 doubles (scanner positions, metres); sid: the station
 * numbers (they select the noise streams).
 * xyz: nst * n_az * n_el x 3 int32 (output); rgb: same rows x 3 uint8, or NULL.
 * Returns 0, or -1 on invalid arguments / allocation failure.
 */
int synth_site(const double* prims_in, int nprim, const double* size, const double* stations,
               const int64_t* sid, int nst, int n_az, int n_el, double sigma, uint64_t seed,
               const double* site_rgb, int32_t* xyz, uint8_t* rgb) {
    if (!prims_in || nprim < 0 || !size || !stations || !sid || nst < 1 || n_az < 1 ||
        n_el < 1 || !xyz)
        return -1;
    prim_t* prims = (prim_t*)malloc(sizeof(prim_t) * (size_t)(nprim > 0 ? nprim : 1));
    if (!prims) return -1;
    for (int q = 0; q < nprim; q++) {
        const double* v = prims_in + 17 * q;
        prim_t* p = &prims[q];
        p->kind = (int)v[0];
        for (int a = 0; a < 3; a++) {
            p->lo[a] = v[1 + a];
            p->hi[a] = v[4 + a];
            p->rgb[a] = v[14 + a];
        }
        p->cx = v[7];
        p->cy = v[8];
        p->r = v[9];
        p->h = v[10];
        p->bcx = v[11];
        p->bcy = v[12];
        p->br = v[13];
    }
    const int64_t per = (int64_t)n_az * n_el;
    const double two_pi = 2.0 * M_PI;
    int rc = 0;
    for (int s = 0; s < nst && !rc; s++) {
        const double* o = stations + 3 * s;
        /* azimuth half-width of each primitive seen from this station (-1: test every ray) */
        double* th = (double*)malloc(sizeof(double) * 2 * (size_t)(nprim > 0 ? nprim : 1));
        if (!th) {
            rc = -1;
            break;
        }
        for (int q = 0; q < nprim; q++) {
            double cx = prims[q].bcx - o[0], cy = prims[q].bcy - o[1];
            double dist = hypot(cx, cy);
            if (dist <= prims[q].br * 1.0001) {
                th[2 * q] = 0.0;
                th[2 * q + 1] = -1.0;
            } else {
                th[2 * q] = atan2(cy, cx);
                th[2 * q + 1] = asin(prims[q].br / dist) + two_pi / n_az;
            }
        }
#pragma omp parallel for schedule(dynamic, 16)
        for (int az = 0; az < n_az; az++) {
            double phi = two_pi * (double)az / (double)n_az;
            double ca = cos(phi), sa = sin(phi);
            int cand[256];
            int nc = 0;
            for (int q = 0; q < nprim && nc < 256; q++) {
                if (th[2 * q + 1] < 0.0) {
                    cand[nc++] = q;
                    continue;
                }
                double dth = remainder(phi - th[2 * q], two_pi);
                if (fabs(dth) <= th[2 * q + 1]) cand[nc++] = q;
            }
            for (int el = 0; el < n_el; el++) {
                double e = -0.5 * M_PI + M_PI * ((double)el + 0.5) / (double)n_el;
                double ce = cos(e), se = sin(e);
                double d[3] = {ca * ce, sa * ce, se};
                int axis;
                double t = box_exit(o, d, size, &axis);
                int hit = -1;
                for (int c = 0; c < nc; c++) {
                    const prim_t* p = &prims[cand[c]];
                    double tt = p->kind == 0 ? box_enter(o, d, p->lo, p->hi) : cyl_enter(o, d, p);
                    if (tt < t) {
                        t = tt;
                        hit = cand[c];
                    }
                }
                int64_t i = (int64_t)az * n_el + el;
                uint64_t st = seed * 0x100000001B3ull ^ ((uint64_t)sid[s] << 40) ^ (uint64_t)i;
                double u1 = unit53(splitmix64(&st)), u2 = unit53(splitmix64(&st));
                double noise = sigma * sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
                double r = t + noise;
                double p[3];
                int64_t row = (int64_t)s * per + i;
                for (int a = 0; a < 3; a++) {
                    p[a] = o[a] + r * d[a];
                    xyz[3 * row + a] = (int32_t)floor(p[a] * 1000.0 + 0.5);
                }
                if (rgb) {
                    const double* base = hit >= 0 ? prims[hit].rgb : site_rgb;
                    long long cell = (long long)floor(p[0] / 0.5) + (long long)floor(p[1] / 0.5) +
                                     (long long)floor(p[2] / 0.5);
                    double f = (cell & 1) ? 0.6 : 1.0;
                    for (int a = 0; a < 3; a++) {
                        double v = base[a] * f;
                        if (v < 0) v = 0;
                        if (v > 255) v = 255;
                        rgb[3 * row + a] = (uint8_t)v;
                    }
                }
            }
        }
        free(th);
    }
    free(prims);
    return rc;
}

int synth_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
