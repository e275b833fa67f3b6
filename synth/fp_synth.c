/*
 * fp_synth.c -- seeded synthetic point clouds (16-byte records: int32 x, y, z,
 * uint8 r, g, b, a).  Holds no octree arithmetic: it only produces inputs, and
 * the CUDA library and the oracle both receive the same bytes from it.
 *
 * Every random number is counter-based: draw k of point i of a cloud with seed
 * s is mix(s * 2^40 + 16 i + k), where mix is the splitmix64 output function
 * (Steele, Lea, Flood 2014).  Points can therefore be generated in any order
 * and by any number of threads with identical bytes.
 *
 *   uniform  x, y, z uniform in [0, 2^bits), r, g, b, a uniform bytes
 *   lidar    500 m x 500 m x 60 m at 1 mm: two-octave gradient-noise terrain
 *            (0..20 m), 200 axis-aligned boxes (walls and roof), 40 scanners
 *            1.8 m above ground; each point picks a scanner, then a surface
 *            element with density falling as 1/r^2 around that scanner
 *            (ground: exact inverse CDF of rho/(rho^2+h^2); boxes: chosen with
 *            weight area/(d^2 + h^2)), then Gaussian jitter sigma = 5 mm
 *            (Box-Muller), quantised and clamped to the scene; RGB from a height
 *            colour ramp plus uniform noise in [-16, 16], alpha = 255.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int32_t x, y, z; uint8_t r, g, b, a; } syn_point;

static inline uint64_t syn_mix(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t seed, uint64_t i, unsigned k)
{
    return syn_mix((seed << 40) + 16 * i + k);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double unit(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------- uniform */
typedef struct {
    uint64_t seed, first, n;
    uint32_t bits;
    syn_point* out;
} uni_job;

static void* uni_run(void* arg)
{
    uni_job* j = (uni_job*)arg;
    uint32_t sh = 64 - j->bits;
    for (uint64_t q = 0; q < j->n; ++q) {
        uint64_t i = j->first + q;
        syn_point p;
        p.x = (int32_t)(draw(j->seed, i, 0) >> sh);
        p.y = (int32_t)(draw(j->seed, i, 1) >> sh);
        p.z = (int32_t)(draw(j->seed, i, 2) >> sh);
        uint64_t c = draw(j->seed, i, 3);
        p.r = (uint8_t)c; p.g = (uint8_t)(c >> 8); p.b = (uint8_t)(c >> 16); p.a = (uint8_t)(c >> 24);
        j->out[q] = p;
    }
    return NULL;
}

/* ---------------------------------------------------------------- lidar */
#define SCENE_X 500000.0
#define SCENE_Y 500000.0
#define SCENE_Z 60000.0
#define N_BOX 200
#define N_SCAN 40
#define SCAN_H 1800.0
#define RHO_MAX 250000.0

typedef struct { double x0, y0, x1, y1, z0, z1; double area[5]; double atotal; } box_t;

typedef struct {
    uint8_t perm[512];
    box_t box[N_BOX];
    double sx[N_SCAN], sy[N_SCAN], sz[N_SCAN];
    double bw[N_SCAN][N_BOX];   /* cumulative box weights per scanner */
    double btotal[N_SCAN];
    double ground_area;         /* weight of the ground per scanner (in the same units) */
} scene_t;

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }

static double grad2(uint8_t h, double x, double y)
{
    switch (h & 7) {
    case 0: return x + y;
    case 1: return -x + y;
    case 2: return x - y;
    case 3: return -x - y;
    case 4: return x;
    case 5: return -x;
    case 6: return y;
    default: return -y;
    }
}

/* 2-D gradient noise with the quintic fade of improved noise; roughly [-1, 1] */
static double noise2(const scene_t* sc, double x, double y)
{
    double fx = floor(x), fy = floor(y);
    int X = (int)fx & 255, Y = (int)fy & 255;
    x -= fx; y -= fy;
    double u = fade(x), v = fade(y);
    const uint8_t* p = sc->perm;
    uint8_t aa = p[p[X] + Y], ab = p[p[X] + Y + 1], ba = p[p[X + 1] + Y], bb = p[p[X + 1] + Y + 1];
    double l0 = grad2(aa, x, y) + u * (grad2(ba, x - 1, y) - grad2(aa, x, y));
    double l1 = grad2(ab, x, y - 1) + u * (grad2(bb, x - 1, y - 1) - grad2(ab, x, y - 1));
    return l0 + v * (l1 - l0);
}

static double terrain(const scene_t* sc, double x, double y)
{
    double n = 0.7 * noise2(sc, x / 100000.0, y / 100000.0) + 0.3 * noise2(sc, x / 25000.0 + 17.0, y / 25000.0 + 31.0);
    double h = 10000.0 + 10000.0 * n;
    if (h < 0.0) h = 0.0;
    if (h > 20000.0) h = 20000.0;
    return h;
}

static void scene_init(scene_t* sc, uint64_t seed)
{
    uint64_t ss = seed ^ 0x5CE4E5CE4E5ull;   /* scene draws use their own stream */
    uint64_t ctr = 0;
    for (int i = 0; i < 256; ++i) sc->perm[i] = (uint8_t)i;
    for (int i = 255; i > 0; --i) {
        int j = (int)(syn_mix((ss << 20) + ctr++) % (uint64_t)(i + 1));
        uint8_t t = sc->perm[i]; sc->perm[i] = sc->perm[j]; sc->perm[j] = t;
    }
    for (int i = 0; i < 256; ++i) sc->perm[256 + i] = sc->perm[i];
    for (int b = 0; b < N_BOX; ++b) {
        box_t* bx = &sc->box[b];
        double cx = unit(syn_mix((ss << 20) + ctr++)) * SCENE_X;
        double cy = unit(syn_mix((ss << 20) + ctr++)) * SCENE_Y;
        double w = 5000.0 + 35000.0 * unit(syn_mix((ss << 20) + ctr++));
        double d = 5000.0 + 35000.0 * unit(syn_mix((ss << 20) + ctr++));
        double h = 4000.0 + 36000.0 * unit(syn_mix((ss << 20) + ctr++));
        bx->x0 = fmax(0.0, cx - w / 2); bx->x1 = fmin(SCENE_X - 1, cx + w / 2);
        bx->y0 = fmax(0.0, cy - d / 2); bx->y1 = fmin(SCENE_Y - 1, cy + d / 2);
        bx->z0 = terrain(sc, cx, cy);
        bx->z1 = fmin(SCENE_Z - 1, bx->z0 + h);
        double W = bx->x1 - bx->x0, D = bx->y1 - bx->y0, H = bx->z1 - bx->z0;
        bx->area[0] = W * H; bx->area[1] = W * H;   /* y0 / y1 walls */
        bx->area[2] = D * H; bx->area[3] = D * H;   /* x0 / x1 walls */
        bx->area[4] = W * D;                        /* roof */
        bx->atotal = 0;
        for (int f = 0; f < 5; ++f) bx->atotal += bx->area[f];
    }
    for (int s = 0; s < N_SCAN; ++s) {
        sc->sx[s] = unit(syn_mix((ss << 20) + ctr++)) * SCENE_X;
        sc->sy[s] = unit(syn_mix((ss << 20) + ctr++)) * SCENE_Y;
        sc->sz[s] = terrain(sc, sc->sx[s], sc->sy[s]) + SCAN_H;
        double acc = 0;
        for (int b = 0; b < N_BOX; ++b) {
            const box_t* bx = &sc->box[b];
            double dx = 0.5 * (bx->x0 + bx->x1) - sc->sx[s];
            double dy = 0.5 * (bx->y0 + bx->y1) - sc->sy[s];
            acc += bx->atotal / (dx * dx + dy * dy + SCAN_H * SCAN_H);
            sc->bw[s][b] = acc;
        }
        sc->btotal[s] = acc;
    }
    /* ground weight: integral of 1/(rho^2+h^2) over the disc, = pi ln(1 + rho_max^2/h^2) */
    sc->ground_area = 3.14159265358979323846 * log(1.0 + RHO_MAX * RHO_MAX / (SCAN_H * SCAN_H));
}

static int clampi(double v, double hi)
{
    if (v < 0.0) v = 0.0;
    if (v > hi) v = hi;
    return (int)v;
}

static uint8_t clampb(int v) { return (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v)); }

typedef struct {
    const scene_t* sc;
    uint64_t seed, first, n;
    syn_point* out;
} lidar_job;

static void* lidar_run(void* arg)
{
    lidar_job* j = (lidar_job*)arg;
    const scene_t* sc = j->sc;
    const double two_pi = 6.28318530717958647692;
    for (uint64_t q = 0; q < j->n; ++q) {
        uint64_t i = j->first + q;
        int s = (int)(draw(j->seed, i, 0) % N_SCAN);
        double u1 = unit(draw(j->seed, i, 1));
        double x, y, z;
        double pb = sc->btotal[s] / (sc->btotal[s] + sc->ground_area);
        if (u1 >= pb) {
            /* ground: rho with density rho/(rho^2+h^2) on [0, RHO_MAX] */
            double L = log(1.0 + RHO_MAX * RHO_MAX / (SCAN_H * SCAN_H));
            double rho = SCAN_H * sqrt(exp(unit(draw(j->seed, i, 2)) * L) - 1.0);
            double th = two_pi * unit(draw(j->seed, i, 3));
            x = sc->sx[s] + rho * cos(th);
            y = sc->sy[s] + rho * sin(th);
            if (x < 0) x = -x;
            if (y < 0) y = -y;
            if (x > SCENE_X - 1) x = 2 * (SCENE_X - 1) - x;
            if (y > SCENE_Y - 1) y = 2 * (SCENE_Y - 1) - y;
            z = terrain(sc, x, y);
        } else {
            /* a box, chosen with weight area / (d^2 + h^2), then a face by area */
            double t = unit(draw(j->seed, i, 2)) * sc->btotal[s];
            int lo = 0, hi = N_BOX - 1;
            while (lo < hi) { int mid = (lo + hi) / 2; if (sc->bw[s][mid] > t) hi = mid; else lo = mid + 1; }
            const box_t* bx = &sc->box[lo];
            double fa = unit(draw(j->seed, i, 3)) * bx->atotal;
            int f = 0;
            while (f < 4 && fa >= bx->area[f]) { fa -= bx->area[f]; ++f; }
            double a = unit(draw(j->seed, i, 4)), b = unit(draw(j->seed, i, 5));
            switch (f) {
            case 0: x = bx->x0 + a * (bx->x1 - bx->x0); y = bx->y0; z = bx->z0 + b * (bx->z1 - bx->z0); break;
            case 1: x = bx->x0 + a * (bx->x1 - bx->x0); y = bx->y1; z = bx->z0 + b * (bx->z1 - bx->z0); break;
            case 2: x = bx->x0; y = bx->y0 + a * (bx->y1 - bx->y0); z = bx->z0 + b * (bx->z1 - bx->z0); break;
            case 3: x = bx->x1; y = bx->y0 + a * (bx->y1 - bx->y0); z = bx->z0 + b * (bx->z1 - bx->z0); break;
            default: x = bx->x0 + a * (bx->x1 - bx->x0); y = bx->y0 + b * (bx->y1 - bx->y0); z = bx->z1; break;
            }
        }
        /* jitter N(0, 5 mm) per axis, Box-Muller */
        double g1 = 1.0 - unit(draw(j->seed, i, 6)), g2 = unit(draw(j->seed, i, 7));
        double g3 = 1.0 - unit(draw(j->seed, i, 8)), g4 = unit(draw(j->seed, i, 9));
        double r1 = sqrt(-2.0 * log(g1)), r2 = sqrt(-2.0 * log(g3));
        x += 5.0 * r1 * cos(two_pi * g2);
        y += 5.0 * r1 * sin(two_pi * g2);
        z += 5.0 * r2 * cos(two_pi * g4);
        syn_point p;
        p.x = clampi(floor(x + 0.5), SCENE_X - 1);
        p.y = clampi(floor(y + 0.5), SCENE_Y - 1);
        p.z = clampi(floor(z + 0.5), SCENE_Z - 1);
        /* height ramp: blue -> green -> yellow -> red over 0..60 m */
        double hz = (double)p.z / SCENE_Z;
        int R, G, B;
        if (hz < 1.0 / 3) { double f = hz * 3; R = 0; G = (int)(255 * f); B = (int)(255 * (1 - f)); }
        else if (hz < 2.0 / 3) { double f = (hz - 1.0 / 3) * 3; R = (int)(255 * f); G = 255; B = 0; }
        else { double f = (hz - 2.0 / 3) * 3; R = 255; G = (int)(255 * (1 - f)); B = 0; }
        uint64_t c = draw(j->seed, i, 10);
        p.r = clampb(R + (int)(c % 33) - 16);
        p.g = clampb(G + (int)((c >> 8) % 33) - 16);
        p.b = clampb(B + (int)((c >> 16) % 33) - 16);
        p.a = 255;
        j->out[q] = p;
    }
    return NULL;
}

/* ------------------------------------------------------------- threads */
typedef void* (*job_fn)(void*);

static void run_threads(job_fn fn, void* jobs, size_t job_size, int nt)
{
    pthread_t th[256];
    int ok[256];
    for (int t = 0; t < nt; ++t) {
        ok[t] = pthread_create(&th[t], NULL, fn, (char*)jobs + (size_t)t * job_size) == 0;
        if (!ok[t]) fn((char*)jobs + (size_t)t * job_size);   /* run inline if no thread */
    }
    for (int t = 0; t < nt; ++t)
        if (ok[t]) pthread_join(th[t], NULL);
}

static int clamp_threads(int nt, uint64_t n)
{
    if (nt < 1) nt = 1;
    if (nt > 256) nt = 256;
    if ((uint64_t)nt > n / 65536 + 1) nt = (int)(n / 65536 + 1);
    return nt;
}

void syn_uniform(uint64_t seed, uint64_t first, uint64_t n, uint32_t bits, void* out, int threads)
{
    int nt = clamp_threads(threads, n);
    uni_job jobs[256];
    uint64_t per = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        uint64_t b = (uint64_t)t * per, e = b + per > n ? n : b + per;
        if (b > n) b = n;
        jobs[t].seed = seed; jobs[t].first = first + b; jobs[t].n = e - b;
        jobs[t].bits = bits; jobs[t].out = (syn_point*)out + b;
    }
    run_threads(uni_run, jobs, sizeof(uni_job), nt);
}

void syn_lidar(uint64_t seed, uint64_t first, uint64_t n, void* out, int threads)
{
    scene_t* sc = (scene_t*)malloc(sizeof(scene_t));
    if (!sc) return;
    scene_init(sc, seed);
    int nt = clamp_threads(threads, n);
    lidar_job jobs[256];
    uint64_t per = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        uint64_t b = (uint64_t)t * per, e = b + per > n ? n : b + per;
        if (b > n) b = n;
        jobs[t].sc = sc; jobs[t].seed = seed; jobs[t].first = first + b; jobs[t].n = e - b;
        jobs[t].out = (syn_point*)out + b;
    }
    run_threads(lidar_run, jobs, sizeof(lidar_job), nt);
    free(sc);
}

/* k-th draw of the size/choice stream of a multi-cloud workload */
uint64_t syn_draw(uint64_t seed, uint64_t i, unsigned k) { return draw(seed, i, k); }
