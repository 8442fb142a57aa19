/*
 * FP64 CPU oracle for differentiable direct volume rendering
 * (Weiss & Westermann, "Differentiable Direct Volume Rendering", Sec. 3-4).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference the CUDA
 * path is checked against. Only the test suite, the package's smoke check and
 * the CPU-baseline leg of the benchmark may load it; the library itself never
 * does, and there is no CPU fallback built on it.
 *
 * It shares no code, header, table or constant generator with the CUDA
 * library. It follows the paper's algorithms in their order and notation:
 *   - ray generation f_camera, sample position x_i = x_o + i*dt*w,
 *     trilinear f_interpolate, transfer function f_TF, front-to-back
 *     f_blend (Alg. 1; Sec. 3.1; Eq. blend-forward),
 *   - the adjoint code in reverse order (Alg. 2; Eq. simpleadjoint), with the
 *     accumulated colour/opacity of every step read from a stored tape
 *     (the "no inversion" scheme of Sec. 4.4), and optionally reconstructed
 *     by the inversion of Eq. inv-blend-forward instead (used only to pin
 *     that the inversion equals the tape),
 *   - forward-mode dual numbers for the three eye coordinates (Sec. 4.2),
 *     an independent derivation of the camera gradient.
 *
 * Readings where the paper is silent (all stated again in the design notes):
 *   - sample emission is premultiplied: C_sample = alpha_i * rgb(d_i), the
 *     Riemann sum of g = tau*C in Eq. 1;
 *   - the printed adjoint of the sample colour, (C - alpha^(i)) C^^(i+1), is
 *     read as (1 - alpha^(i)) C^^(i+1) (derivative of Eq. blend-forward);
 *   - TF control point r sits at density r/(R-1); d is clamped to [0,1]
 *     (zero derivative outside); k = min(floor(d(R-1)), R-2);
 *   - grid vertices at -ext/2 + j*h, h = 1/(max(n)-1), box centred at 0;
 *   - absorption-only model: tau = d, output opacity A = 1 - exp(-sum dt d);
 *   - x_o is the entry into the box, N = ceil(L/dt - 2^-10);
 *   - the ray setup (frame, slab test, N) is evaluated with every operation
 *     rounded to binary32 when fp32 != 0, because the kernel decides the
 *     integer N in that precision; everything after it is binary64.
 *
 * Parity pins (tests/test_oracle.py): Beer-Lambert closed form, constant-TF
 * closed form, exact trilinear reproduction of linear fields, dot-product
 * (transpose) identity of the absorption projector, central finite
 * differences of every parameter on 8^3 volumes, dual numbers vs tape,
 * inversion vs tape.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_ABSORPTION 0
#define ORA_EMISSION_ABSORPTION 1
#define ORA_COLOR_VOLUME 2      /* pre-shaded (r, g, b, tau) per vertex, Sec. 5.4 */

/* Shape of the grid and the discretisation of the ray (Sec. 3.1). */
typedef struct {
    int n[3];          /* nx, ny, nz */
    double half[3];    /* half extent of the box along each axis */
    double inv_h;      /* grid units per world unit, max(n) - 1 */
    double dt;         /* step in world units */
    int vf32;          /* volume samples stored as float (else double) */
} grid_t;

/* density of vertex i (float samples are widened exactly) */
static inline double vget(const void* V, const grid_t* G, long i)
{
    return G->vf32 ? (double)((const float*)V)[i] : ((const double*)V)[i];
}

/* Camera of one view. */
typedef struct {
    int width, height, ortho;
    double lens;       /* tan(fov_y/2) (perspective) or image height (ortho) */
    double eye[3];
} cam_t;

/* Everything f_camera produces for one pixel, kept for the adjoint. */
typedef struct {
    int N, axis, degenerate;
    double o[3], w[3], xo[3];
    double tn, tfar, q;
    double f[3], r[3], u[3];
    double el, ql, dl, su, sv;
} ray_t;

static inline double rnd(int fp32, double x) { return fp32 ? (double)(float)x : x; }

static void make_grid(int nx, int ny, int nz, double step, int fp32, grid_t* G)
{
    G->n[0] = nx; G->n[1] = ny; G->n[2] = nz;
    G->vf32 = 0;
    int nm = nx > ny ? nx : ny;
    if (nz > nm) nm = nz;
    G->inv_h = (double)(nm - 1);
    G->dt = rnd(fp32, step / (double)(nm - 1));
    for (int a = 0; a < 3; ++a)
        G->half[a] = rnd(fp32, rnd(fp32, (double)(G->n[a] - 1) / (double)(nm - 1)) * 0.5);
}

/*
 * f_camera (Alg. 1, second line): origin and unit direction of the ray
 * through pixel (px, py), clipped against the volume box.
 * The camera sits at `eye`, looks at the box centre, world up is +y
 * (right vector fixed to +x when looking straight along y).
 * Every operation goes through R_ so that with fp32 != 0 each result is the
 * correctly rounded binary32 value of the same expression.
 */
static void camera_ray(const cam_t* c, const grid_t* G, int px, int py, int fp32, ray_t* r)
{
#define R_(x) rnd(fp32, (x))
    const double* e = c->eye;
    double e2 = R_(R_(R_(e[0] * e[0]) + R_(e[1] * e[1])) + R_(e[2] * e[2]));
    r->el = R_(sqrt(e2));
    for (int a = 0; a < 3; ++a) r->f[a] = R_(-e[a] / r->el);
    double q2 = R_(R_(r->f[0] * r->f[0]) + R_(r->f[2] * r->f[2]));
    if (q2 < 0x1p-26) {
        r->degenerate = 1;
        r->ql = 0.0;
        r->r[0] = 1.0; r->r[1] = 0.0; r->r[2] = 0.0;
    } else {
        r->degenerate = 0;
        r->ql = R_(sqrt(q2));
        r->r[0] = R_(-r->f[2] / r->ql);
        r->r[1] = 0.0;
        r->r[2] = R_(r->f[0] / r->ql);
    }
    /* up = right x forward */
    r->u[0] = R_(R_(r->r[1] * r->f[2]) - R_(r->r[2] * r->f[1]));
    r->u[1] = R_(R_(r->r[2] * r->f[0]) - R_(r->r[0] * r->f[2]));
    r->u[2] = R_(R_(r->r[0] * r->f[1]) - R_(r->r[1] * r->f[0]));

    double sx = R_(R_((double)(2 * px + 1) / (double)c->width) - 1.0);
    double sy = R_(1.0 - R_((double)(2 * py + 1) / (double)c->height));
    double aspect = R_((double)c->width / (double)c->height);
    if (!c->ortho) {
        r->su = R_(sx * R_(c->lens * aspect));
        r->sv = R_(sy * c->lens);
        double d[3];
        for (int a = 0; a < 3; ++a)
            d[a] = R_(R_(r->f[a] + R_(r->su * r->r[a])) + R_(r->sv * r->u[a]));
        r->dl = R_(sqrt(R_(R_(R_(d[0] * d[0]) + R_(d[1] * d[1])) + R_(d[2] * d[2]))));
        for (int a = 0; a < 3; ++a) {
            r->w[a] = R_(d[a] / r->dl);
            r->o[a] = e[a];
        }
    } else {
        double hh = R_(c->lens * 0.5);
        r->su = R_(sx * R_(hh * aspect));
        r->sv = R_(sy * hh);
        r->dl = 1.0;
        for (int a = 0; a < 3; ++a) {
            r->o[a] = R_(R_(e[a] + R_(r->su * r->r[a])) + R_(r->sv * r->u[a]));
            r->w[a] = r->f[a];
        }
    }

    /* slab test against [-half, half]^3; entry clamped to the camera */
    double tn = 0.0, tfar = INFINITY;
    int axis = -1, hit = 1;
    for (int a = 0; a < 3; ++a) {
        if (r->w[a] != 0.0) {
            double t0 = R_(R_(-G->half[a] - r->o[a]) / r->w[a]);
            double t1 = R_(R_(G->half[a] - r->o[a]) / r->w[a]);
            double tnear = t0 < t1 ? t0 : t1;
            double tfr = t0 < t1 ? t1 : t0;
            if (tnear > tn) { tn = tnear; axis = a; }
            if (tfr < tfar) tfar = tfr;
        } else if (r->o[a] < -G->half[a] || r->o[a] > G->half[a]) {
            hit = 0;
        }
    }
    r->tn = tn;
    r->tfar = tfar;
    r->axis = axis;
    r->N = 0;
    r->q = 0.0;
    if (hit && tfar > tn) {
        double L = R_(tfar - tn);
        r->q = R_(L / G->dt);
        double nq = ceil(R_(r->q - 0x1p-10));
        r->N = nq > 0.0 ? (int)nq : 0;
    }
    for (int a = 0; a < 3; ++a) r->xo[a] = R_(r->o[a] + R_(tn * r->w[a]));
#undef R_
}

/*
 * f_interpolate (Alg. 1; Sec. 3.1): trilinear interpolation of the vertex
 * densities at world position x. Fills the 8 corner indices and weights and
 * the derivative of the density w.r.t. the grid coordinate (zero along an
 * axis where x was clamped to the box).
 */
static double interpolate_strided(const void* V, const grid_t* G, const double x[3], int stride, int ch,
                                  long idx[8], double wt[8], double dg[3]);

static double interpolate(const void* V, const grid_t* G, const double x[3],
                          long idx[8], double wt[8], double dg[3])
{
    return interpolate_strided(V, G, x, 1, 0, idx, wt, dg);
}

/* The same for channel `ch` of a volume with `stride` values per vertex
 * (vertex idx holds V[idx*stride .. idx*stride+stride-1]). */
static double interpolate_strided(const void* V, const grid_t* G, const double x[3], int stride, int ch,
                                  long idx[8], double wt[8], double dg[3])
{
    int j[3];
    double fr[3];
    int inside[3];
    for (int a = 0; a < 3; ++a) {
        double g = (x[a] + G->half[a]) * G->inv_h;
        inside[a] = 1;
        if (g < 0.0) { g = 0.0; inside[a] = 0; }
        if (g > (double)(G->n[a] - 1)) { g = (double)(G->n[a] - 1); inside[a] = 0; }
        int jj = (int)floor(g);
        if (jj > G->n[a] - 2) jj = G->n[a] - 2;
        j[a] = jj;
        fr[a] = g - (double)jj;
    }
    double d = 0.0;
    double val[8];
    for (int c = 0; c < 8; ++c) {
        int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        idx[c] = ((long)(j[2] + cz) * G->n[1] + (j[1] + cy)) * (long)G->n[0] + (j[0] + cx);
        wt[c] = (cx ? fr[0] : 1.0 - fr[0]) * (cy ? fr[1] : 1.0 - fr[1]) * (cz ? fr[2] : 1.0 - fr[2]);
        val[c] = vget(V, G, idx[c] * stride + ch);
        d += wt[c] * val[c];
    }
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int c = 0; c < 8; ++c) {
            int b[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
            double p = b[a] ? 1.0 : -1.0;   /* d/dfr_a of the corner weight */
            for (int o = 0; o < 3; ++o)
                if (o != a) p *= b[o] ? fr[o] : 1.0 - fr[o];
            s += p * val[c];
        }
        dg[a] = inside[a] ? s : 0.0;
    }
    return d;
}

/*
 * f_TF (Alg. 1; Sec. 3.1): R regularly spaced control points, control point
 * r at density r/(R-1), linear in between; d clamped to [0,1].
 * out = (r, g, b, tau). *k, *fr give the interpolated segment; *slope is 0
 * when d was clamped.
 */
static void transfer(const double* tf, int R, double d, double out[4], int* k, double* fr, int* slope)
{
    double dc = d;
    *slope = 1;
    if (dc < 0.0) { dc = 0.0; *slope = 0; }
    if (dc > 1.0) { dc = 1.0; *slope = 0; }
    double u = dc * (double)(R - 1);
    int kk = (int)floor(u);
    if (kk > R - 2) kk = R - 2;
    *k = kk;
    *fr = u - (double)kk;
    for (int ch = 0; ch < 4; ++ch)
        out[ch] = (1.0 - *fr) * tf[4 * kk + ch] + *fr * tf[4 * (kk + 1) + ch];
}

typedef struct {
    const void* V;
    const double* tf;
    int R, model;
    grid_t G;
    cam_t cam;
} scene_t;

/* One sample i of the ray (positions, interpolation, TF). */
typedef struct {
    double x[3], d, c[4], tau, alpha;
    long idx[8];
    double wt[8], dg[3];
    double dg4[4][3];   /* colour volume: d(channel)/d(grid coordinate) */
    int k, slope;
    double fr;
    double ge;        /* binary32 error bound of the grid coordinates (ambiguity bounds only) */
} sample_t;

static double grid_error(const void* smp, const grid_t* G, double margin)
{
    const sample_t* sm = (const sample_t*)smp;
    double gmax = 1.0;
    for (int a = 0; a < 3; ++a) {
        double g = fabs((sm->x[a] + G->half[a]) * G->inv_h);
        if (g > gmax) gmax = g;
    }
    return margin * ldexp(1.0, ilogb(gmax) - 23);
}

static double density_error(const void* smp, const void* V, const grid_t* G, double margin)
{
    const sample_t* sm = (const sample_t*)smp;
    double vmax = 0.0, gsum = 0.0;
    for (int c = 0; c < 8; ++c)
        if (fabs(vget(V, G, sm->idx[c])) > vmax) vmax = fabs(vget(V, G, sm->idx[c]));
    for (int a = 0; a < 3; ++a) gsum += fabs(sm->dg[a]);
    return gsum * sm->ge + margin * 4.0 * 0x1p-24 * vmax;
}

static void eval_sample(const scene_t* s, const ray_t* ry, int i, sample_t* sm)
{
    double ti = (double)i * s->G.dt;
    for (int a = 0; a < 3; ++a) sm->x[a] = ry->xo[a] + ti * ry->w[a];
    if (s->model == ORA_COLOR_VOLUME) {
        /* Sec. 5.4: the volume holds (r, g, b, tau) per vertex, no TF */
        for (int ch = 0; ch < 4; ++ch)
            sm->c[ch] = interpolate_strided(s->V, &s->G, sm->x, 4, ch, sm->idx, sm->wt, sm->dg4[ch]);
        sm->d = sm->c[3];
        sm->tau = sm->c[3];
        sm->k = 0; sm->fr = 0.0; sm->slope = 1;
        for (int a = 0; a < 3; ++a) sm->dg[a] = sm->dg4[3][a];
        sm->alpha = 1.0 - exp(-s->G.dt * sm->tau);
        return;
    }
    sm->d = interpolate(s->V, &s->G, sm->x, sm->idx, sm->wt, sm->dg);
    if (s->model == ORA_EMISSION_ABSORPTION) {
        transfer(s->tf, s->R, sm->d, sm->c, &sm->k, &sm->fr, &sm->slope);
        sm->tau = sm->c[3];
    } else {
        sm->c[0] = sm->c[1] = sm->c[2] = 0.0;
        sm->tau = sm->d;
        sm->c[3] = sm->d;
        sm->k = 0; sm->fr = 0.0; sm->slope = 1;
    }
    /* Beer-Lambert segment opacity */
    sm->alpha = 1.0 - exp(-s->G.dt * sm->tau);
}

/*
 * Alg. 1 for one ray. State (C, A) is the accumulated premultiplied colour
 * and opacity, blended front to back per Eq. blend-forward. When `tapeA` /
 * `tapeC` are given, the state before every step is stored (the O(N) tape).
 * Returns the optical depth S = sum dt*tau (used by the transpose pin).
 */
static double march(const scene_t* s, const ray_t* ry, double out[4], double* tapeA, double* tapeC)
{
    double C[3] = {0.0, 0.0, 0.0}, A = 0.0, S = 0.0;
    sample_t sm;
    for (int i = 0; i < ry->N; ++i) {
        if (tapeA) {
            tapeA[i] = A;
            for (int ch = 0; ch < 3; ++ch) tapeC[3 * i + ch] = C[ch];
        }
        eval_sample(s, ry, i, &sm);
        for (int ch = 0; ch < 3; ++ch) C[ch] = C[ch] + (1.0 - A) * (sm.alpha * sm.c[ch]);
        A = A + (1.0 - A) * sm.alpha;
        S += s->G.dt * sm.tau;
    }
    if (tapeA) {
        tapeA[ry->N] = A;
        for (int ch = 0; ch < 3; ++ch) tapeC[3 * ry->N + ch] = C[ch];
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = A;
    return S;
}

static void setup_scene(scene_t* s, const void* V, int vf32, int nx, int ny, int nz, const double* tf,
                        int R, int model, int W, int H, int ortho, double lens, const double* eye,
                        double step, int fp32)
{
    s->V = V; s->tf = tf; s->R = R; s->model = model;
    make_grid(nx, ny, nz, step, fp32, &s->G);
    s->G.vf32 = vf32;
    s->cam.width = W; s->cam.height = H; s->cam.ortho = ortho; s->cam.lens = lens;
    for (int a = 0; a < 3; ++a) s->cam.eye[a] = eye[a];
}

static int channels(int model) { return model == ORA_ABSORPTION ? 1 : 4; }

/*
 * Forward render of one view. `pix` lists the linear pixel indices to
 * evaluate (NULL = all W*H in order). Outputs per listed pixel: image
 * (4 channels RGBA, or 1 channel A for the absorption model), the sample
 * count N and the optical depth S.
 */
int ora_render(const void* V, int vf32, int nx, int ny, int nz, const double* tf, int R, int model,
               int W, int H, int ortho, double lens, const double* eye, double step, int fp32,
               const int64_t* pix, int64_t npix, double* image, int32_t* nsamp, double* depth)
{
    scene_t s;
    setup_scene(&s, V, vf32, nx, ny, nz, tf, R, model, W, H, ortho, lens, eye, step, fp32);
    int64_t total = pix ? npix : (int64_t)W * H;
    int nc = channels(model);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < total; ++t) {
        int64_t p = pix ? pix[t] : t;
        ray_t ry;
        camera_ray(&s.cam, &s.G, (int)(p % W), (int)(p / W), fp32, &ry);
        double out[4];
        double S = march(&s, &ry, out, NULL, NULL);
        if (nc == 4) for (int ch = 0; ch < 4; ++ch) image[4 * t + ch] = out[ch];
        else image[t] = out[3];
        if (nsamp) nsamp[t] = ry.N;
        if (depth) depth[t] = S;
    }
    return 0;
}

/* Per-pixel ray description: N, q = L/dt, tn, tfar, x_o, w. */
int ora_rays(int nx, int ny, int nz, int W, int H, int ortho, double lens, const double* eye,
             double step, int fp32, int32_t* nsamp, double* q, double* geo /* [W*H][8] */)
{
    scene_t s;
    setup_scene(&s, NULL, 0, nx, ny, nz, NULL, 2, 0, W, H, ortho, lens, eye, step, fp32);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < (int64_t)W * H; ++p) {
        ray_t ry;
        camera_ray(&s.cam, &s.G, (int)(p % W), (int)(p / W), fp32, &ry);
        nsamp[p] = ry.N;
        if (q) q[p] = ry.q;
        if (geo) {
            geo[8 * p + 0] = ry.tn; geo[8 * p + 1] = ry.tfar;
            for (int a = 0; a < 3; ++a) { geo[8 * p + 2 + a] = ry.xo[a]; geo[8 * p + 5 + a] = ry.w[a]; }
        }
    }
    return 0;
}

/* Trilinear density at world points x[n][3] (for the linear-field pin). */
int ora_interpolate(const double* V, int nx, int ny, int nz, const double* x, int64_t n, double* d)
{
    grid_t G;
    make_grid(nx, ny, nz, 1.0, 0, &G);
    for (int64_t t = 0; t < n; ++t) {
        long idx[8]; double wt[8], dg[3];
        d[t] = interpolate(V, &G, x + 3 * t, idx, wt, dg);
    }
    return 0;
}

/*
 * For each axis a where the grid coordinate of x lies within `delta` of an
 * integer (a face between two cells, or a box face where the coordinate is
 * clamped), the jump of d(density)/d(g_a) across that face; 0 elsewhere.
 */
static void face_jumps_strided(const void* V, const grid_t* G, const double x[3], double delta, int stride,
                               int chn, double jump[3]);

static void face_jumps(const void* V, const grid_t* G, const double x[3], double delta, double jump[3])
{
    face_jumps_strided(V, G, x, delta, 1, 0, jump);
}

static void face_jumps_strided(const void* V, const grid_t* G, const double x[3], double delta, int stride,
                               int chn, double jump[3])
{
    double g[3];
    for (int a = 0; a < 3; ++a) g[a] = (x[a] + G->half[a]) * G->inv_h;
    for (int a = 0; a < 3; ++a) {
        jump[a] = 0.0;
        double f = floor(g[a] + 0.5);
        if (fabs(g[a] - f) >= delta) continue;
        int face = (int)f;            /* vertex index of the face along axis a */
        double slope[2];              /* normal derivative in cells face-1 and face */
        for (int sd = 0; sd < 2; ++sd) {
            int cell = face - 1 + sd;
            if (cell < 0 || cell > G->n[a] - 2) { slope[sd] = 0.0; continue; }
            /* other two axes: trilinear weights at x (clamped) */
            double pt[3] = {x[0], x[1], x[2]};
            int j[3];
            double fr[3];
            for (int b = 0; b < 3; ++b) {
                double gb = (pt[b] + G->half[b]) * G->inv_h;
                if (gb < 0.0) gb = 0.0;
                if (gb > (double)(G->n[b] - 1)) gb = (double)(G->n[b] - 1);
                int jj = (int)floor(gb);
                if (jj > G->n[b] - 2) jj = G->n[b] - 2;
                j[b] = jj;
                fr[b] = gb - (double)jj;
            }
            j[a] = cell;
            double sum = 0.0;
            for (int c = 0; c < 8; ++c) {
                int bb[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
                double w = bb[a] ? 1.0 : -1.0;
                for (int o = 0; o < 3; ++o)
                    if (o != a) w *= bb[o] ? fr[o] : 1.0 - fr[o];
                long idx = ((long)(j[2] + bb[2]) * G->n[1] + (j[1] + bb[1])) * (long)G->n[0] + (j[0] + bb[0]);
                sum += w * vget(V, G, idx * stride + chn);
            }
            slope[sd] = sum;
        }
        jump[a] = fabs(slope[1] - slope[0]);
    }
}

/* binary32 error bound of a sample's grid coordinates: one ulp of the
 * largest coordinate (times margin). */
static double grid_error(const void* smp, const grid_t* G, double margin);
/* binary32 error bound of a sample's density. */
static double density_error(const void* smp, const void* V, const grid_t* G, double margin);

static inline void atomic_add(double* p, double v)
{
#pragma omp atomic
    *p += v;
}

static inline void atomic_miss(int64_t* n)
{
#pragma omp atomic
    *n += 1;
}

/*
 * Adjoint of f_camera: chain the adjoints of the entry point x_o and the
 * direction w back to the eye position (last line of Alg. 2's loop body
 * and the f_camera line after it). Covers the dependence of the entry
 * distance tn on origin and direction through the slab face that set it.
 */
static void camera_adjoint(const cam_t* c, const ray_t* r, const double xo_hat[3],
                           const double w_hat_in[3], double e_hat[3])
{
    double xw = xo_hat[0] * r->w[0] + xo_hat[1] * r->w[1] + xo_hat[2] * r->w[2];
    double o_hat[3], w_hat[3];
    for (int a = 0; a < 3; ++a) {
        o_hat[a] = xo_hat[a];
        w_hat[a] = w_hat_in[a] + r->tn * xo_hat[a];
    }
    if (r->axis >= 0) {
        int a = r->axis;
        o_hat[a] += -xw / r->w[a];
        w_hat[a] += -r->tn / r->w[a] * xw;
    }
    double f_hat[3] = {0, 0, 0}, r_hat[3] = {0, 0, 0}, u_hat[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) e_hat[a] = o_hat[a];
    if (!c->ortho) {
        double ww = r->w[0] * w_hat[0] + r->w[1] * w_hat[1] + r->w[2] * w_hat[2];
        for (int a = 0; a < 3; ++a) {
            double dh = (w_hat[a] - r->w[a] * ww) / r->dl;
            f_hat[a] += dh;
            r_hat[a] += r->su * dh;
            u_hat[a] += r->sv * dh;
        }
    } else {
        for (int a = 0; a < 3; ++a) {
            r_hat[a] += r->su * o_hat[a];
            u_hat[a] += r->sv * o_hat[a];
            f_hat[a] += w_hat[a];
        }
    }
    /* up = r x f */
    r_hat[0] += r->f[1] * u_hat[2] - r->f[2] * u_hat[1];
    r_hat[1] += r->f[2] * u_hat[0] - r->f[0] * u_hat[2];
    r_hat[2] += r->f[0] * u_hat[1] - r->f[1] * u_hat[0];
    f_hat[0] += u_hat[1] * r->r[2] - u_hat[2] * r->r[1];
    f_hat[1] += u_hat[2] * r->r[0] - u_hat[0] * r->r[2];
    f_hat[2] += u_hat[0] * r->r[1] - u_hat[1] * r->r[0];
    /* r = q/|q|, q = (-f_z, 0, f_x) */
    if (!r->degenerate) {
        double rr = r->r[0] * r_hat[0] + r->r[1] * r_hat[1] + r->r[2] * r_hat[2];
        double q_hat[3];
        for (int a = 0; a < 3; ++a) q_hat[a] = (r_hat[a] - r->r[a] * rr) / r->ql;
        f_hat[2] += -q_hat[0];
        f_hat[0] += q_hat[2];
    }
    /* f = -e/|e| */
    double ff = r->f[0] * f_hat[0] + r->f[1] * f_hat[1] + r->f[2] * f_hat[2];
    for (int a = 0; a < 3; ++a) e_hat[a] += -(f_hat[a] - r->f[a] * ff) / r->el;
}

/*
 * Adjoint pass (Alg. 2) for one view, summed over the listed pixels.
 * grad_image holds dL/d(image) per listed pixel (4 or 1 channels).
 * Gradients are ADDED to grad_vol [nz][ny][nx], grad_tf [R][4],
 * grad_eye [3] and grad_step [1]; any may be NULL.
 * invert = 0: the state (A_i, C_i) before each step is read from the tape.
 * invert = 1: it is reconstructed from (A_{i+1}, C_{i+1}) with
 *             Eq. inv-blend-forward (paper's alpha form).
 */
/*
 * margin > 0: ambiguity bounds for a binary32 evaluation of the same
 * samples. f_TF is piecewise linear, so d(f_TF)/dd jumps at every control
 * point (and at the clamp ends 0 and 1), and the normal derivative of the
 * trilinear density jumps at every cell face. A binary32 evaluation puts
 * the grid coordinate g within one ulp of max|g| (the double-float sample
 * positions round twice by half an ulp), the density within |grad d| times
 * that plus four ulps of the largest corner value, and u = d (R-1) within
 * one more ulp; `margin` multiplies these error bounds. A sample closer to
 * a kink than its bound may legitimately take either one-sided derivative:
 *   amb_vol: w_c * |d^_left - d^_right| summed at its 8 corners (TF kinks);
 *   amb_eye: the change of x^_i from either kind of kink, chained through
 *            the camera adjoint, summed in absolute value.
 */
/*
 * Where the volume gradient of vertex `idx` is stored: at idx itself
 * (dense output), or, with a selection `sel` (ascending vertex indices),
 * at its position in `sel` (compact output for volumes whose dense
 * binary64 gradient would not fit in host memory); -1 if the vertex is not
 * selected (counted by the caller as a miss).
 */
typedef struct {
    const int64_t* sel;
    int64_t n;
} vsel_t;

static inline int64_t vslot(const vsel_t* vs, long idx)
{
    if (!vs->sel) return idx;
    int64_t lo = 0, hi = vs->n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (vs->sel[mid] == idx) return mid;
        if (vs->sel[mid] < idx) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static int64_t backward_impl(const void* V, int vf32, int nx, int ny, int nz, const double* tf, int R, int model,
                         int W, int H, int ortho, double lens, const double* eye, double step, int fp32,
                         const int64_t* pix, int64_t npix, const double* grad_image, int invert,
                         double* grad_vol, double* grad_tf, double* grad_eye, double* grad_step,
                         double margin, double* amb_vol, double* amb_eye, const vsel_t* vs);

int ora_backward(const void* V, int vf32, int nx, int ny, int nz, const double* tf, int R, int model,
                 int W, int H, int ortho, double lens, const double* eye, double step, int fp32,
                 const int64_t* pix, int64_t npix, const double* grad_image, int invert,
                 double* grad_vol, double* grad_tf, double* grad_eye, double* grad_step,
                 double margin, double* amb_vol, double* amb_eye)
{
    vsel_t vs = {NULL, 0};
    return (int)backward_impl(V, vf32, nx, ny, nz, tf, R, model, W, H, ortho, lens, eye, step, fp32, pix, npix,
                         grad_image, invert, grad_vol, grad_tf, grad_eye, grad_step, margin, amb_vol, amb_eye,
                         &vs);
}

/*
 * ora_backward with the volume gradient (and its kink bound) stored
 * compactly: grad_vol[k] (grad_vol[4k + ch] for colour volumes) and
 * amb_vol[k] belong to vertex sel[k], sel ascending. Returns the number of
 * vertex contributions that found no slot (0 when sel lists every vertex
 * the rays touch, as ora_touched gives).
 */
int64_t ora_backward_sel(const void* V, int vf32, int nx, int ny, int nz, const double* tf, int R, int model,
                         int W, int H, int ortho, double lens, const double* eye, double step, int fp32,
                         const int64_t* pix, int64_t npix, const double* grad_image, int invert,
                         double* grad_vol, double* grad_tf, double* grad_eye, double* grad_step,
                         double margin, double* amb_vol, double* amb_eye, const int64_t* sel, int64_t nsel)
{
    vsel_t vs = {sel, nsel};
    return backward_impl(V, vf32, nx, ny, nz, tf, R, model, W, H, ortho, lens, eye, step, fp32, pix, npix,
                         grad_image, invert, grad_vol, grad_tf, grad_eye, grad_step, margin, amb_vol, amb_eye,
                         &vs);
}

/*
 * The 8 corner vertices of every sample of the listed rays (Alg. 1's
 * f_interpolate footprint), in march order, duplicates included. With
 * out == NULL only counts them. Returns the count (or, with out given, the
 * number written, at most cap).
 */
int64_t ora_touched(int nx, int ny, int nz, int W, int H, int ortho, double lens, const double* eye,
                    double step, int fp32, const int64_t* pix, int64_t npix, int64_t* out, int64_t cap)
{
    scene_t s;
    setup_scene(&s, NULL, 0, nx, ny, nz, NULL, 2, ORA_ABSORPTION, W, H, ortho, lens, eye, step, fp32);
    int64_t total = pix ? npix : (int64_t)W * H;
    int64_t k = 0;
    for (int64_t t = 0; t < total; ++t) {
        int64_t p = pix ? pix[t] : t;
        ray_t ry;
        camera_ray(&s.cam, &s.G, (int)(p % W), (int)(p / W), fp32, &ry);
        for (int i = 0; i < ry.N; ++i) {
            double x[3];
            double ti = (double)i * s.G.dt;
            for (int a = 0; a < 3; ++a) x[a] = ry.xo[a] + ti * ry.w[a];
            /* the corner indices of f_interpolate at x (values not read) */
            int j[3];
            for (int a = 0; a < 3; ++a) {
                double g = (x[a] + s.G.half[a]) * s.G.inv_h;
                if (g < 0.0) g = 0.0;
                if (g > (double)(s.G.n[a] - 1)) g = (double)(s.G.n[a] - 1);
                int jj = (int)floor(g);
                if (jj > s.G.n[a] - 2) jj = s.G.n[a] - 2;
                j[a] = jj;
            }
            for (int c = 0; c < 8; ++c) {
                if (out && k >= cap) return k;
                if (out)
                    out[k] = ((long)(j[2] + ((c >> 2) & 1)) * s.G.n[1] + (j[1] + ((c >> 1) & 1))) * (long)s.G.n[0]
                             + (j[0] + (c & 1));
                ++k;
            }
        }
    }
    return k;
}

static int64_t backward_impl(const void* V, int vf32, int nx, int ny, int nz, const double* tf, int R, int model,
                         int W, int H, int ortho, double lens, const double* eye, double step, int fp32,
                         const int64_t* pix, int64_t npix, const double* grad_image, int invert,
                         double* grad_vol, double* grad_tf, double* grad_eye, double* grad_step,
                         double margin, double* amb_vol, double* amb_eye, const vsel_t* vs)
{
    int64_t misses = 0;
    scene_t s;
    setup_scene(&s, V, vf32, nx, ny, nz, tf, R, model, W, H, ortho, lens, eye, step, fp32);
    int64_t total = pix ? npix : (int64_t)W * H;
    int nc = channels(model);
    const double dt = s.G.dt;
#pragma omp parallel
    {
        double eye_acc[3] = {0, 0, 0}, step_acc = 0.0, amb_acc[3] = {0, 0, 0};
        /* per-thread TF sums, added to grad_tf once at the end */
        double* tf_acc = grad_tf ? (double*)calloc((size_t)4 * R, sizeof(double)) : NULL;
        double* tapeA = NULL;
        double* tapeC = NULL;
        int cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < total; ++t) {
            int64_t p = pix ? pix[t] : t;
            ray_t ry;
            camera_ray(&s.cam, &s.G, (int)(p % W), (int)(p / W), fp32, &ry);
            if (ry.N == 0) continue;
            if (ry.N + 1 > cap) {
                cap = ry.N + 1;
                tapeA = (double*)realloc(tapeA, sizeof(double) * cap);
                tapeC = (double*)realloc(tapeC, sizeof(double) * 3 * cap);
            }
            double out[4];
            march(&s, &ry, out, tapeA, tapeC);

            /* seed: colour_N^ from dL/d(image) (first line of Alg. 2) */
            double Ch[3] = {0, 0, 0}, Ah;
            if (nc == 4) {
                for (int ch = 0; ch < 3; ++ch) Ch[ch] = grad_image[4 * t + ch];
                Ah = grad_image[4 * t + 3];
            } else {
                Ah = grad_image[t];
            }
            double A1 = tapeA[ry.N], C1[3] = {tapeC[3 * ry.N], tapeC[3 * ry.N + 1], tapeC[3 * ry.N + 2]};
            double xo_hat[3] = {0, 0, 0}, w_hat[3] = {0, 0, 0}, dt_hat = 0.0;
            sample_t sm;
            for (int i = ry.N - 1; i >= 0; --i) {
                eval_sample(&s, &ry, i, &sm);
                sm.ge = margin > 0.0 ? grid_error(&sm, &s.G, margin) : 0.0;
                double A0, C0[3];
                double Cs[3];
                for (int ch = 0; ch < 3; ++ch) Cs[ch] = sm.alpha * sm.c[ch];
                if (!invert) {
                    A0 = tapeA[i];
                    for (int ch = 0; ch < 3; ++ch) C0[ch] = tapeC[3 * i + ch];
                } else {
                    /* Eq. inv-blend-forward */
                    A0 = (sm.alpha - A1) / (sm.alpha - 1.0);
                    for (int ch = 0; ch < 3; ++ch) C0[ch] = C1[ch] - (1.0 - A0) * Cs[ch];
                }
                /* Eq. adj-blend-forward: adjoints of the sample (alpha, C_s)
                 * and of the state before the step; C^ is unchanged. */
                double CsC = Cs[0] * Ch[0] + Cs[1] * Ch[1] + Cs[2] * Ch[2];
                double a_hat = (1.0 - A0) * Ah;
                double Cs_hat[3];
                for (int ch = 0; ch < 3; ++ch) Cs_hat[ch] = (1.0 - A0) * Ch[ch];
                Ah = (1.0 - sm.alpha) * Ah - CsC;
                /* premultiplication C_s = alpha * rgb */
                double c_hat[4];
                for (int ch = 0; ch < 3; ++ch) {
                    c_hat[ch] = sm.alpha * Cs_hat[ch];
                    a_hat += sm.c[ch] * Cs_hat[ch];
                }
                /* alpha = 1 - exp(-dt tau) */
                double e = 1.0 - sm.alpha;
                double tau_hat = a_hat * dt * e;
                dt_hat += a_hat * sm.tau * e;
                c_hat[3] = tau_hat;
                /* f_TF adjoint */
                double d_hat, d_jump = 0.0;
                if (model == ORA_EMISSION_ABSORPTION) {
                    if (tf_acc) {
                        for (int ch = 0; ch < 4; ++ch) {
                            tf_acc[4 * sm.k + ch] += (1.0 - sm.fr) * c_hat[ch];
                            tf_acc[4 * (sm.k + 1) + ch] += sm.fr * c_hat[ch];
                        }
                    }
                    d_hat = 0.0;
                    if (sm.slope)
                        for (int ch = 0; ch < 4; ++ch)
                            d_hat += (double)(R - 1) * (tf[4 * (sm.k + 1) + ch] - tf[4 * sm.k + ch]) * c_hat[ch];
                    if ((amb_vol || amb_eye) && margin > 0.0) {
                        double u = sm.d * (double)(R - 1);
                        double kn = floor(u + 0.5);
                        double eu = (R - 1) * density_error(&sm, V, &s.G, margin) + margin * 0x1p-23 * fabs(u);
                        if (kn >= 0.0 && kn <= (double)(R - 1) && fabs(u - kn) < eu) {
                            int knot = (int)kn;
                            double side[2] = {0.0, 0.0};   /* segments knot-1 and knot */
                            for (int sd = 0; sd < 2; ++sd) {
                                int seg = knot - 1 + sd;
                                if (seg < 0 || seg > R - 2) continue;
                                for (int ch = 0; ch < 4; ++ch)
                                    side[sd] += (double)(R - 1) * (tf[4 * (seg + 1) + ch] - tf[4 * seg + ch]) * c_hat[ch];
                            }
                            double jump = fabs(side[1] - side[0]);
                            d_jump = jump;
                            if (amb_vol)
                                for (int c = 0; c < 8; ++c) {
                                    int64_t q = vslot(vs, sm.idx[c]);
                                    if (q < 0) { atomic_miss(&misses); continue; }
                                    atomic_add(&amb_vol[q], sm.wt[c] * jump);
                                }
                        }
                    }
                } else {
                    d_hat = tau_hat;
                }
                /* f_interpolate adjoint; gd = d(L)/d(grid coordinate) */
                double gd[3];
                if (model == ORA_COLOR_VOLUME) {
                    if (grad_vol)
                        for (int c = 0; c < 8; ++c) {
                            int64_t q = vslot(vs, sm.idx[c]);
                            if (q < 0) { atomic_miss(&misses); continue; }
                            for (int ch = 0; ch < 4; ++ch)
                                atomic_add(&grad_vol[q * 4 + ch], sm.wt[c] * c_hat[ch]);
                        }
                    for (int a = 0; a < 3; ++a) {
                        gd[a] = 0.0;
                        for (int ch = 0; ch < 4; ++ch) gd[a] += sm.dg4[ch][a] * c_hat[ch];
                    }
                } else {
                    if (grad_vol)
                        for (int c = 0; c < 8; ++c) {
                            int64_t q = vslot(vs, sm.idx[c]);
                            if (q < 0) { atomic_miss(&misses); continue; }
                            atomic_add(&grad_vol[q], sm.wt[c] * d_hat);
                        }
                    for (int a = 0; a < 3; ++a) gd[a] = sm.dg[a] * d_hat;
                }
                double ti = (double)i * dt;
                double xi_w = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double x_hat = gd[a] * s.G.inv_h;
                    xo_hat[a] += x_hat;
                    w_hat[a] += ti * x_hat;
                    xi_w += (double)i * ry.w[a] * x_hat;
                }
                dt_hat += xi_w;
                if (amb_eye && margin > 0.0) {
                    /* change of x^_i if the TF kink or a cell face is taken
                     * from the other side */
                    double dx[3];
                    int any = 0;
                    double dgn[3];
                    if (model == ORA_COLOR_VOLUME) {
                        for (int a = 0; a < 3; ++a) dx[a] = 0.0;
                        for (int ch = 0; ch < 4; ++ch) {
                            face_jumps_strided(V, &s.G, sm.x, sm.ge, 4, ch, dgn);
                            for (int a = 0; a < 3; ++a) dx[a] += fabs(dgn[a] * c_hat[ch]) * s.G.inv_h;
                        }
                        for (int a = 0; a < 3; ++a) any |= dx[a] != 0.0;
                    } else {
                        face_jumps(V, &s.G, sm.x, sm.ge, dgn);
                        for (int a = 0; a < 3; ++a) {
                            dx[a] = (fabs(sm.dg[a] * d_jump) + fabs(dgn[a] * d_hat)) * s.G.inv_h;
                            any |= dx[a] != 0.0;
                        }
                    }
                    if (any) {
                        /* the camera adjoint is linear: bound each axis' part */
                        for (int a = 0; a < 3; ++a) {
                            if (dx[a] == 0.0) continue;
                            double xo1[3] = {0, 0, 0}, w1[3] = {0, 0, 0}, eh[3];
                            xo1[a] = dx[a];
                            w1[a] = ti * dx[a];
                            camera_adjoint(&s.cam, &ry, xo1, w1, eh);
                            for (int b = 0; b < 3; ++b) amb_acc[b] += fabs(eh[b]);
                        }
                    }
                }
                A1 = A0;
                for (int ch = 0; ch < 3; ++ch) C1[ch] = C0[ch];
            }
            if (grad_eye) {
                double eh[3];
                camera_adjoint(&s.cam, &ry, xo_hat, w_hat, eh);
                for (int a = 0; a < 3; ++a) eye_acc[a] += eh[a];
            }
            step_acc += dt_hat;
        }
        if (grad_eye)
            for (int a = 0; a < 3; ++a) atomic_add(&grad_eye[a], eye_acc[a]);
        if (amb_eye)
            for (int a = 0; a < 3; ++a) atomic_add(&amb_eye[a], amb_acc[a]);
        if (tf_acc) {
            for (int j = 0; j < 4 * R; ++j) atomic_add(&grad_tf[j], tf_acc[j]);
            free(tf_acc);
        }
        /* dt = step/(max(n)-1) */
        if (grad_step) atomic_add(grad_step, step_acc / s.G.inv_h);
        free(tapeA);
        free(tapeC);
    }
    return misses;
}

/* ---------------------------------------------------------------------- */
/* Forward-mode differentiation w.r.t. the eye position (Sec. 4.2).        */
/* A dual number carries a value and its derivatives w.r.t. eye x, y, z.   */
/* ---------------------------------------------------------------------- */
typedef struct { double v, d[3]; } dual;

static inline dual dc(double v) { dual r = {v, {0, 0, 0}}; return r; }
static inline dual dadd(dual a, dual b) { dual r; r.v = a.v + b.v; for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
static inline dual dsub(dual a, dual b) { dual r; r.v = a.v - b.v; for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
static inline dual dmul(dual a, dual b) { dual r; r.v = a.v * b.v; for (int k = 0; k < 3; ++k) r.d[k] = a.v * b.d[k] + b.v * a.d[k]; return r; }
static inline dual ddiv(dual a, dual b) { dual r; r.v = a.v / b.v; for (int k = 0; k < 3; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v); return r; }
static inline dual dsqrt(dual a) { dual r; r.v = sqrt(a.v); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] / (2.0 * r.v); return r; }
static inline dual dexp(dual a) { dual r; r.v = exp(a.v); for (int k = 0; k < 3; ++k) r.d[k] = r.v * a.d[k]; return r; }
static inline dual dneg(dual a) { dual r; r.v = -a.v; for (int k = 0; k < 3; ++k) r.d[k] = -a.d[k]; return r; }

/*
 * Forward render of one view with dual numbers seeded on the eye position.
 * Ray setup in binary64 (the integer N and the slab face are taken from the
 * values). Outputs image [npix][nc] and dimage [npix][nc][3].
 */
int ora_render_dual(const void* V, int vf32, int nx, int ny, int nz, const double* tf, int R, int model,
                    int W, int H, int ortho, double lens, const double* eye, double step, int n_fp32,
                    const int64_t* pix, int64_t npix, double* image, double* dimage)
{
    scene_t s;
    setup_scene(&s, V, vf32, nx, ny, nz, tf, R, model, W, H, ortho, lens, eye, step, 0);
    const grid_t* G = &s.G;
    int64_t total = pix ? npix : (int64_t)W * H;
    int nc = channels(model);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < total; ++t) {
        int64_t p = pix ? pix[t] : t;
        int px = (int)(p % W), py = (int)(p / W);
        dual e[3];
        for (int a = 0; a < 3; ++a) { e[a] = dc(eye[a]); e[a].d[a] = 1.0; }
        dual el = dsqrt(dadd(dadd(dmul(e[0], e[0]), dmul(e[1], e[1])), dmul(e[2], e[2])));
        dual f[3], r[3], u[3];
        for (int a = 0; a < 3; ++a) f[a] = ddiv(dneg(e[a]), el);
        double q2 = f[0].v * f[0].v + f[2].v * f[2].v;
        if (q2 < 0x1p-26) {
            r[0] = dc(1.0); r[1] = dc(0.0); r[2] = dc(0.0);
        } else {
            dual ql = dsqrt(dadd(dmul(f[0], f[0]), dmul(f[2], f[2])));
            r[0] = ddiv(dneg(f[2]), ql); r[1] = dc(0.0); r[2] = ddiv(f[0], ql);
        }
        u[0] = dsub(dmul(r[1], f[2]), dmul(r[2], f[1]));
        u[1] = dsub(dmul(r[2], f[0]), dmul(r[0], f[2]));
        u[2] = dsub(dmul(r[0], f[1]), dmul(r[1], f[0]));
        double sx = (double)(2 * px + 1) / W - 1.0;
        double sy = 1.0 - (double)(2 * py + 1) / H;
        double aspect = (double)W / H;
        dual o[3], w[3];
        if (!ortho) {
            double su = sx * lens * aspect, sv = sy * lens;
            dual d[3];
            for (int a = 0; a < 3; ++a) d[a] = dadd(dadd(f[a], dmul(dc(su), r[a])), dmul(dc(sv), u[a]));
            dual dl = dsqrt(dadd(dadd(dmul(d[0], d[0]), dmul(d[1], d[1])), dmul(d[2], d[2])));
            for (int a = 0; a < 3; ++a) { w[a] = ddiv(d[a], dl); o[a] = e[a]; }
        } else {
            double hh = lens * 0.5, su = sx * hh * aspect, sv = sy * hh;
            for (int a = 0; a < 3; ++a) {
                o[a] = dadd(dadd(e[a], dmul(dc(su), r[a])), dmul(dc(sv), u[a]));
                w[a] = f[a];
            }
        }
        dual tn = dc(0.0);
        double tfar = INFINITY;
        int hit = 1;
        for (int a = 0; a < 3; ++a) {
            if (w[a].v != 0.0) {
                dual t0 = ddiv(dsub(dc(-G->half[a]), o[a]), w[a]);
                dual t1 = ddiv(dsub(dc(G->half[a]), o[a]), w[a]);
                dual tnear = t0.v < t1.v ? t0 : t1;
                double tfr = t0.v < t1.v ? t1.v : t0.v;
                if (tnear.v > tn.v) tn = tnear;
                if (tfr < tfar) tfar = tfr;
            } else if (o[a].v < -G->half[a] || o[a].v > G->half[a]) {
                hit = 0;
            }
        }
        int N = 0;
        if (hit && tfar > tn.v) {
            double nq = ceil((tfar - tn.v) / G->dt - 0x1p-10);
            N = nq > 0.0 ? (int)nq : 0;
        }
        if (n_fp32) {
            /* take the integer N from the binary32 setup of the kernel (the
             * derivatives stay binary64) */
            scene_t s32;
            setup_scene(&s32, V, vf32, nx, ny, nz, tf, R, model, W, H, ortho, lens, eye, step, 1);
            ray_t r32;
            camera_ray(&s32.cam, &s32.G, px, py, 1, &r32);
            N = r32.N;
        }
        dual xo[3];
        for (int a = 0; a < 3; ++a) xo[a] = dadd(o[a], dmul(tn, w[a]));

        dual C[3] = {dc(0), dc(0), dc(0)}, A = dc(0);
        for (int i = 0; i < N; ++i) {
            /* x_i = x_o + i dt w, grid coordinate, trilinear weights */
            dual fr[3];
            int j[3], inside[3];
            for (int a = 0; a < 3; ++a) {
                dual x = dadd(xo[a], dmul(dc((double)i * G->dt), w[a]));
                dual g = dmul(dadd(x, dc(G->half[a])), dc(G->inv_h));
                inside[a] = 1;
                if (g.v < 0.0) { g = dc(0.0); inside[a] = 0; }
                if (g.v > (double)(G->n[a] - 1)) { g = dc((double)(G->n[a] - 1)); inside[a] = 0; }
                int jj = (int)floor(g.v);
                if (jj > G->n[a] - 2) jj = G->n[a] - 2;
                j[a] = jj;
                fr[a] = dsub(g, dc((double)jj));
                (void)inside[a];
            }
            dual d = dc(0.0);
            for (int c = 0; c < 8; ++c) {
                int b[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
                dual wt = dc(1.0);
                for (int a = 0; a < 3; ++a) wt = dmul(wt, b[a] ? fr[a] : dsub(dc(1.0), fr[a]));
                long idx = ((long)(j[2] + b[2]) * G->n[1] + (j[1] + b[1])) * (long)G->n[0] + (j[0] + b[0]);
                d = dadd(d, dmul(wt, dc(vget(V, G, idx))));
            }
            dual col[4];
            if (model == ORA_COLOR_VOLUME) {
                for (int ch = 0; ch < 4; ++ch) {
                    col[ch] = dc(0.0);
                    for (int c = 0; c < 8; ++c) {
                        int b[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
                        dual wt = dc(1.0);
                        for (int a = 0; a < 3; ++a) wt = dmul(wt, b[a] ? fr[a] : dsub(dc(1.0), fr[a]));
                        long idx = ((long)(j[2] + b[2]) * G->n[1] + (j[1] + b[1])) * (long)G->n[0] + (j[0] + b[0]);
                        col[ch] = dadd(col[ch], dmul(wt, dc(vget(V, G, idx * 4 + ch))));
                    }
                }
            } else if (model == ORA_EMISSION_ABSORPTION) {
                dual dcl = d;
                if (dcl.v < 0.0) dcl = dc(0.0);
                if (dcl.v > 1.0) dcl = dc(1.0);
                dual uu = dmul(dcl, dc((double)(R - 1)));
                int k = (int)floor(uu.v);
                if (k > R - 2) k = R - 2;
                dual frt = dsub(uu, dc((double)k));
                for (int ch = 0; ch < 4; ++ch)
                    col[ch] = dadd(dmul(dsub(dc(1.0), frt), dc(tf[4 * k + ch])), dmul(frt, dc(tf[4 * (k + 1) + ch])));
            } else {
                col[0] = col[1] = col[2] = dc(0.0);
                col[3] = d;
            }
            dual alpha = dsub(dc(1.0), dexp(dmul(dc(-G->dt), col[3])));
            dual T = dsub(dc(1.0), A);
            for (int ch = 0; ch < 3; ++ch) C[ch] = dadd(C[ch], dmul(T, dmul(alpha, col[ch])));
            A = dadd(A, dmul(T, alpha));
        }
        if (nc == 4) {
            for (int ch = 0; ch < 3; ++ch) {
                image[4 * t + ch] = C[ch].v;
                for (int k = 0; k < 3; ++k) dimage[(4 * t + ch) * 3 + k] = C[ch].d[k];
            }
            image[4 * t + 3] = A.v;
            for (int k = 0; k < 3; ++k) dimage[(4 * t + 3) * 3 + k] = A.d[k];
        } else {
            image[t] = A.v;
            for (int k = 0; k < 3; ++k) dimage[t * 3 + k] = A.d[k];
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Orbit camera: eye on a sphere from longitude (yaw), latitude (pitch)    */
/* and distance (Sec. 5.1: "parameterized by longitude and latitude").     */
/* e = dist * (cos p sin y, sin p, cos p cos y); yaw = pitch = 0 is +z.    */
/* ---------------------------------------------------------------------- */
int ora_orbit_eye(const double* params, int64_t n, double* eye)
{
    for (int64_t v = 0; v < n; ++v) {
        double y = params[3 * v], p = params[3 * v + 1], dist = params[3 * v + 2];
        eye[3 * v + 0] = dist * cos(p) * sin(y);
        eye[3 * v + 1] = dist * sin(p);
        eye[3 * v + 2] = dist * cos(p) * cos(y);
    }
    return 0;
}

int ora_orbit_eye_backward(const double* params, int64_t n, const double* grad_eye, double* grad_params)
{
    for (int64_t v = 0; v < n; ++v) {
        double y = params[3 * v], p = params[3 * v + 1], dist = params[3 * v + 2];
        const double* g = grad_eye + 3 * v;
        double dy[3] = {dist * cos(p) * cos(y), 0.0, -dist * cos(p) * sin(y)};
        double dp[3] = {-dist * sin(p) * sin(y), dist * cos(p), -dist * sin(p) * cos(y)};
        double dd[3] = {cos(p) * sin(y), sin(p), cos(p) * cos(y)};
        grad_params[3 * v + 0] += g[0] * dy[0] + g[1] * dy[1] + g[2] * dy[2];
        grad_params[3 * v + 1] += g[0] * dp[0] + g[1] * dp[1] + g[2] * dp[2];
        grad_params[3 * v + 2] += g[0] * dd[0] + g[1] * dd[1] + g[2] * dd[2];
    }
    return 0;
}

int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
