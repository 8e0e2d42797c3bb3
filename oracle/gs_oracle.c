/*
 * gs_oracle.c -- FP64 CPU oracle for batched 3D Gaussian Splatting rendering.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code, header,
 * table or constant with the CUDA path, and it never reads anything the CUDA
 * path produced.
 *
 * What it computes: the renderer the paper drops into its vectorised simulator
 * (Sec. 3.2 "3D Gaussian Splatting as a Drop-in Renderer"; Fig. 4: depth is a
 * by-product of the same compositing pass), i.e. the 3DGS rasteriser it cites
 * (Sec. 2.3, a scene as a set of oriented 3D Gaussians), with these constants:
 * EWA projection with a 0.3 px dilation, 3-sigma tile culling, 16x16 tiles,
 * per-tile order by (depth, Gaussian index), alpha = min(0.99, o*exp(power)),
 * alpha < 1/255 skipped, stop before T would fall below 1e-4. Every step is
 * done literally in double precision; nothing is blocked, fused or reordered.
 *
 * Readings where the paper is silent (it only cites the rasteriser):
 *  - quaternion order (w, x, y, z), normalised before use;
 *  - viewmat is world->camera, OpenCV axes (x right, y down, z forward);
 *  - pixel (i, j) has its centre at (i + 0.5, j + 0.5);
 *  - near plane 0.2, no far plane;
 *  - Jacobian guard band: x/z clamped to [-(cx + g'W/2)/fx, (W - cx + g'W/2)/fx]
 *    with g' = guard - 1 (= the symmetric 1.3 tan(fov/2) clamp when cx = W/2);
 *  - radius r = sigma * sqrt(lambda_max), no rounding;
 *  - tile rect: inclusive [max(0, floor((u-r)/16)), min(TX-1, floor((u+r)/16))],
 *    culled if u+r < 0, u-r >= W, v+r < 0 or v-r >= H;
 *  - SH: real basis with the Condon-Shortley phase, coefficients l-major with
 *    m = -l..l, view direction = camera centre -> mean in world coordinates,
 *    colour = max(0, 0.5 + sum c*Y), no upper clamp;
 *  - depth D = sum_i w_i z_i with z the camera-space depth of the mean,
 *    background 0 for depth, bg colour for rgb (C + T*bg);
 *  - the Gaussian whose T(1-alpha) would fall below T_min is not added.
 *
 * Near-threshold decisions. A float32 implementation may take either branch of
 * a decision whose double-precision operands lie within a small band of the
 * threshold (tile membership at a rect edge or the cull boundary, the near
 * plane, the order of two Gaussians of almost equal depth, alpha at 1/255, T at
 * T_min). The bands are parameters; with all bands zero the oracle is the plain
 * definition. With bands > 0 the renderer reports, for each pixel whose primary
 * (double) walk met such a decision, the results of the walks that flip up to
 * `max_flips` of those decisions, so a test can accept any of them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* prm[]: rendering constants */
enum { P_NEAR, P_DIL, P_GUARD, P_SIGMA, P_AMIN, P_AMAX, P_TMIN, P_BG0, P_BG1, P_BG2, P_TILE,
       P_COUNT };
/* band[]: near-threshold bands (all zero = plain definition) */
enum { B_PX_ABS, B_PX_REL, B_Z_ABS, B_Z_REL, B_LNA, B_T_REL, B_MAXFLIP, B_MAXLEAF, B_COUNT };
/* per-Gaussian projected record */
enum { R_U, R_V, R_Z, R_O, R_CA, R_CB, R_CC, R_RAD, R_SA, R_SB, R_SC, R_RED, R_GRN, R_BLU,
       R_PX, R_PY, R_LMAX, R_DET, R_COUNT = 20 };
/* per-Gaussian status bits */
#define ST_VALID 1 /* survives every cull in double precision */
#define ST_AMBIG 2 /* the near-plane or off-image cull lies within the band */
#define ST_PROJ 4  /* a record was computed (z > 0 and z > near or near-ambiguous) */

int or_abi_version(void) { return 3; }

/* ---------------------------------------------------------------- SH basis */

static double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* Associated Legendre function P_l^m(x), m >= 0, Condon-Shortley phase, by the
 * textbook three-term recurrence in l starting from P_m^m and P_{m+1}^m. */
static double assoc_legendre(int l, int m, double x) {
    double pmm = 1.0;
    if (m > 0) {
        double s = sqrt((1.0 - x) * (1.0 + x));
        double odd = 1.0;
        for (int i = 1; i <= m; ++i) {
            pmm *= -odd * s;
            odd += 2.0;
        }
    }
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pl = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pl = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (double)(ll - m);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

/* Real spherical harmonics Y_lm(dir) for l <= deg, written l-major, m = -l..l:
 *   m > 0: sqrt(2) K_lm cos(m phi) P_l^m(cos theta)
 *   m = 0: K_l0 P_l^0(cos theta)
 *   m < 0: sqrt(2) K_l|m| sin(|m| phi) P_l^|m|(cos theta)
 * with K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), theta measured from +z and
 * phi = atan2(y, x). dir must be a unit vector. */
void or_sh_basis(int deg, double x, double y, double z, double *out) {
    double phi = atan2(y, x);
    int k = 0;
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            double P = assoc_legendre(l, am, z);
            double v;
            if (m == 0)
                v = K * P;
            else if (m > 0)
                v = sqrt(2.0) * K * cos(m * phi) * P;
            else
                v = sqrt(2.0) * K * sin(am * phi) * P;
            out[k++] = v;
        }
    }
}

/* ------------------------------------------------------- Gaussian geometry */

/* Rotation matrix (row-major) of the normalised quaternion (w, x, y, z). */
void or_quat_to_rot(const double *q_in, double *R) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = 1.0, x = 0.0, y = 0.0, z = 0.0;
    if (n > 0.0) {
        w = q_in[0] / n;
        x = q_in[1] / n;
        y = q_in[2] / n;
        z = q_in[3] / n;
    }
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* World-space covariance Sigma = R S S^T R^T, S = diag(exp(log_scale)). */
void or_cov3d(const double *log_scale, const double *q, double *Sig) {
    double R[9], M[9];
    or_quat_to_rot(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * exp(log_scale[j]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += M[3 * i + k] * M[3 * j + k];
            Sig[3 * i + j] = s;
        }
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------ camera */

typedef struct {
    double R[9], t[3], fx, fy, cx, cy, cpos[3];
    double lim_xp, lim_xn, lim_yp, lim_yn;
    int W, H, TX, TY, tile;
} ocam;

static void make_cam(const double *vm, const double *intr, int W, int H, const double *prm,
                     ocam *c) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) c->R[3 * i + j] = vm[4 * i + j];
        c->t[i] = vm[4 * i + 3];
    }
    c->fx = intr[0];
    c->fy = intr[1];
    c->cx = intr[2];
    c->cy = intr[3];
    /* camera centre in the world: C = -R^T t */
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i) s += c->R[3 * i + j] * c->t[i];
        c->cpos[j] = -s;
    }
    double g = prm[P_GUARD] - 1.0;
    c->lim_xp = ((W - c->cx) + g * 0.5 * W) / c->fx;
    c->lim_xn = (c->cx + g * 0.5 * W) / c->fx;
    c->lim_yp = ((H - c->cy) + g * 0.5 * H) / c->fy;
    c->lim_yn = (c->cy + g * 0.5 * H) / c->fy;
    c->W = W;
    c->H = H;
    c->tile = (int)prm[P_TILE];
    c->TX = (W + c->tile - 1) / c->tile;
    c->TY = (H + c->tile - 1) / c->tile;
}

/* Tile rect of the pixel interval [lo_x, hi_x] x [lo_y, hi_y]; empty (x0 > x1)
 * when the interval lies off the image. */
static void rect_of(double lo_x, double hi_x, double lo_y, double hi_y, const ocam *c, int *r) {
    r[0] = 1;
    r[1] = 0;
    r[2] = 1;
    r[3] = 0;
    if (lo_x > hi_x || lo_y > hi_y) return;
    if (hi_x < 0.0 || lo_x >= (double)c->W || hi_y < 0.0 || lo_y >= (double)c->H) return;
    double ts = (double)c->tile;
    int x0 = (int)floor(lo_x / ts), x1 = (int)floor(hi_x / ts);
    int y0 = (int)floor(lo_y / ts), y1 = (int)floor(hi_y / ts);
    r[0] = x0 < 0 ? 0 : x0;
    r[1] = x1 > c->TX - 1 ? c->TX - 1 : x1;
    r[2] = y0 < 0 ? 0 : y0;
    r[3] = y1 > c->TY - 1 ? c->TY - 1 : y1;
}

static int rect_has(const int *r, int tx, int ty) {
    return tx >= r[0] && tx <= r[1] && ty >= r[2] && ty <= r[3];
}

typedef struct {
    const double *mean, *log_scale, *quat, *logit, *sh;
    int64_t n;
    int deg;
} oscene;

/* Project Gaussian g for camera c (EWA splatting, the cited 3DGS projection):
 *   p = R_c mu + t_c;  cull z <= near
 *   J = [[fx/z, 0, -fx x~/z^2], [0, fy/z, -fy y~/z^2]] with x~, y~ the
 *       guard-band-clamped x, y;  Sigma' = J R_c Sigma R_c^T J^T + dil I
 *   conic = inverse(Sigma'), r = sigma sqrt(lambda_max(Sigma'))
 *   u = fx x/z + cx, v = fy y/z + cy; tile rect; SH colour.
 * Writes rec (R_COUNT doubles) and three rects: primary, ext (bounds widened by
 * the pixel band), inner (bounds shrunk by it). Returns the status bits. */
static int project_one(const oscene *s, int64_t g, const ocam *c, const double *prm,
                       const double *band, double *rec, int *rect, int *ext, int *inner) {
    memset(rec, 0, sizeof(double) * R_COUNT);
    for (int i = 0; i < 4; ++i) rect[i] = ext[i] = inner[i] = (i & 1) ? 0 : 1;
    double mu[3] = {s->mean[g], s->mean[s->n + g], s->mean[2 * s->n + g]};
    double p[3];
    for (int i = 0; i < 3; ++i)
        p[i] = c->R[3 * i] * mu[0] + c->R[3 * i + 1] * mu[1] + c->R[3 * i + 2] * mu[2] + c->t[i];
    double z = p[2];
    double bz = band[B_Z_ABS] + band[B_Z_REL] * fabs(z);
    int near_amb = fabs(z - prm[P_NEAR]) <= bz && bz > 0.0;
    if (!(z > prm[P_NEAR]) && !near_amb) return 0;
    if (!(z > 0.0)) return 0;
    int st = ST_PROJ;
    if (z > prm[P_NEAR]) st |= ST_VALID;
    if (near_amb) st |= ST_AMBIG;

    double ls[3] = {s->log_scale[g], s->log_scale[s->n + g], s->log_scale[2 * s->n + g]};
    double q[4] = {s->quat[g], s->quat[s->n + g], s->quat[2 * s->n + g], s->quat[3 * s->n + g]};
    double Sig[9];
    or_cov3d(ls, q, Sig);

    double xz = p[0] / z, yz = p[1] / z;
    double xc = xz < -c->lim_xn ? -c->lim_xn : (xz > c->lim_xp ? c->lim_xp : xz);
    double yc = yz < -c->lim_yn ? -c->lim_yn : (yz > c->lim_yp ? c->lim_yp : yz);
    double tx = xc * z, ty = yc * z;
    double J[6] = {c->fx / z, 0.0, -c->fx * tx / (z * z), 0.0, c->fy / z, -c->fy * ty / (z * z)};
    double T[6]; /* T = J R_c, 2x3 */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += J[3 * i + k] * c->R[3 * k + j];
            T[3 * i + j] = acc;
        }
    double TS[6]; /* T Sigma */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += T[3 * i + k] * Sig[3 * k + j];
            TS[3 * i + j] = acc;
        }
    double cov[4]; /* T Sigma T^T */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += TS[3 * i + k] * T[3 * j + k];
            cov[2 * i + j] = acc;
        }
    double a = cov[0] + prm[P_DIL], b = cov[1], cc = cov[3] + prm[P_DIL];
    double det = a * cc - b * b;
    if (!(det > 0.0)) return 0;
    double mid = 0.5 * (a + cc);
    double disc = mid * mid - det;
    double lmax = mid + sqrt(disc > 0.0 ? disc : 0.0);
    double r = prm[P_SIGMA] * sqrt(lmax);
    double u = c->fx * xz + c->cx, v = c->fy * yz + c->cy;

    rec[R_U] = u;
    rec[R_V] = v;
    rec[R_Z] = z;
    rec[R_O] = sigmoid(s->logit[g]);
    rec[R_CA] = cc / det;
    rec[R_CB] = -b / det;
    rec[R_CC] = a / det;
    rec[R_RAD] = r;
    rec[R_SA] = a;
    rec[R_SB] = b;
    rec[R_SC] = cc;
    rec[R_PX] = p[0];
    rec[R_PY] = p[1];
    rec[R_LMAX] = lmax;
    rec[R_DET] = det;

    rect_of(u - r, u + r, v - r, v + r, c, rect);
    if (rect[0] > rect[1]) st &= ~ST_VALID;
    double bp = band[B_PX_ABS] + band[B_PX_REL] * (fabs(u) + fabs(v) + r);
    rect_of(u - r - bp, u + r + bp, v - r - bp, v + r + bp, c, ext);
    rect_of(u - r + bp, u + r - bp, v - r + bp, v + r - bp, c, inner);
    if (bp > 0.0) {
        /* off-image cull within the band of its boundary */
        if (fabs(u + r) <= bp || fabs(u - r - c->W) <= bp || fabs(v + r) <= bp ||
            fabs(v - r - c->H) <= bp)
            st |= ST_AMBIG;
    }

    /* view-dependent colour */
    double d[3] = {mu[0] - c->cpos[0], mu[1] - c->cpos[1], mu[2] - c->cpos[2]};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double Y[16];
    if (dn > 0.0)
        or_sh_basis(s->deg, d[0] / dn, d[1] / dn, d[2] / dn, Y);
    else
        or_sh_basis(s->deg, 0.0, 0.0, 1.0, Y);
    int K = (s->deg + 1) * (s->deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += s->sh[((int64_t)k * 3 + ch) * s->n + g] * Y[k];
        rec[R_RED + ch] = acc > 0.0 ? acc : 0.0;
    }
    return st;
}

/* Public: project every Gaussian of a scene for one camera.
 * mean[3N], log_scale[3N], quat[4N] (w,x,y,z rows), logit[N], sh[K*3*N]
 * (coefficient-major, then channel, then Gaussian), viewmat[16] row-major,
 * intr[4] = fx, fy, cx, cy. Outputs: rec[N*R_COUNT], rects[N*12] (primary,
 * ext, inner as x0,x1,y0,y1), status[N]. Returns the number of valid ones. */
int64_t or_project(int64_t n, int deg, const double *mean, const double *log_scale,
                   const double *quat, const double *logit, const double *sh,
                   const double *viewmat, const double *intr, int W, int H, const double *prm,
                   const double *band, double *rec, int32_t *rects, int32_t *status) {
    oscene s = {mean, log_scale, quat, logit, sh, n, deg};
    ocam c;
    make_cam(viewmat, intr, W, H, prm, &c);
    int64_t nvalid = 0;
#pragma omp parallel for schedule(static) reduction(+ : nvalid)
    for (int64_t g = 0; g < n; ++g) {
        int r0[4], r1[4], r2[4];
        int st = project_one(&s, g, &c, prm, band, rec + g * R_COUNT, r0, r1, r2);
        for (int i = 0; i < 4; ++i) {
            rects[g * 12 + i] = r0[i];
            rects[g * 12 + 4 + i] = r1[i];
            rects[g * 12 + 8 + i] = r2[i];
        }
        status[g] = st;
        nvalid += (st & ST_VALID) ? 1 : 0;
    }
    return nvalid;
}

/* ------------------------------------------------------------- tile lists */

typedef struct {
    int64_t g;
    double z;
    unsigned char prim;  /* member in the double-precision decision */
    unsigned char amb;   /* membership lies within the band */
    unsigned char zswap; /* depth within the band of the next entry's */
} oent;

static int ent_cmp(const void *pa, const void *pb) {
    const oent *a = (const oent *)pa, *b = (const oent *)pb;
    if (a->z < b->z) return -1;
    if (a->z > b->z) return 1;
    return (a->g > b->g) - (a->g < b->g);
}

typedef struct {
    double *rec;
    int32_t *rects;
    int32_t *status;
    int64_t *off; /* [ntiles+1] */
    oent *ent;    /* extended lists, each sorted by (z, g) */
    int ntiles;
} olists;

/* Build, for every tile, the extended list: all Gaussians whose widened rect
 * contains the tile, sorted by (z, index), with membership / ambiguity flags.
 * With zero bands the extended list is exactly the tile's list. */
static int build_lists(const oscene *s, const ocam *c, const double *prm, const double *band,
                       olists *L) {
    int64_t n = s->n;
    L->ntiles = c->TX * c->TY;
    L->rec = (double *)malloc(sizeof(double) * R_COUNT * (n > 0 ? n : 1));
    L->rects = (int32_t *)malloc(sizeof(int32_t) * 12 * (n > 0 ? n : 1));
    L->status = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    L->off = (int64_t *)calloc((size_t)L->ntiles + 1, sizeof(int64_t));
    L->ent = NULL;
    if (!L->rec || !L->rects || !L->status || !L->off) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        int r0[4], r1[4], r2[4];
        int st = project_one(s, g, c, prm, band, L->rec + g * R_COUNT, r0, r1, r2);
        for (int i = 0; i < 4; ++i) {
            L->rects[g * 12 + i] = r0[i];
            L->rects[g * 12 + 4 + i] = r1[i];
            L->rects[g * 12 + 8 + i] = r2[i];
        }
        L->status[g] = st;
    }
    /* count entries per tile (serial: exact and simple) */
    int64_t *cnt = (int64_t *)calloc((size_t)L->ntiles, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t g = 0; g < n; ++g) {
        if (!(L->status[g] & ST_PROJ)) continue;
        const int32_t *e = L->rects + g * 12 + 4;
        for (int ty = e[2]; ty <= e[3]; ++ty)
            for (int tx = e[0]; tx <= e[1]; ++tx) cnt[ty * c->TX + tx]++;
    }
    for (int t = 0; t < L->ntiles; ++t) L->off[t + 1] = L->off[t] + cnt[t];
    int64_t total = L->off[L->ntiles];
    L->ent = (oent *)malloc(sizeof(oent) * (total > 0 ? total : 1));
    if (!L->ent) {
        free(cnt);
        return -1;
    }
    for (int t = 0; t < L->ntiles; ++t) cnt[t] = L->off[t];
    for (int64_t g = 0; g < n; ++g) {
        int st = L->status[g];
        if (!(st & ST_PROJ)) continue;
        const int32_t *r0 = L->rects + g * 12, *e = L->rects + g * 12 + 4,
                      *in = L->rects + g * 12 + 8;
        for (int ty = e[2]; ty <= e[3]; ++ty)
            for (int tx = e[0]; tx <= e[1]; ++tx) {
                oent *E = &L->ent[cnt[ty * c->TX + tx]++];
                E->g = g;
                E->z = L->rec[g * R_COUNT + R_Z];
                E->prim = (st & ST_VALID) && rect_has(r0, tx, ty);
                /* every entry lies in the widened rect: a member is certain only
                 * when the shrunk rect still holds the tile, and a non-member here
                 * could become one under a perturbation within the band */
                int certain = (st & ST_VALID) && !(st & ST_AMBIG) && rect_has(in, tx, ty);
                E->amb = (unsigned char)!certain;
                E->zswap = 0;
            }
    }
    free(cnt);
    double bz_abs = band[B_Z_ABS], bz_rel = band[B_Z_REL];
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < L->ntiles; ++t) {
        oent *E = L->ent + L->off[t];
        int64_t m = L->off[t + 1] - L->off[t];
        qsort(E, (size_t)m, sizeof(oent), ent_cmp);
        if (bz_abs > 0.0 || bz_rel > 0.0)
            for (int64_t k = 0; k + 1 < m; ++k) {
                double dz = fabs(E[k + 1].z - E[k].z);
                if (dz <= bz_abs + bz_rel * fabs(E[k].z)) E[k].zswap = 1;
            }
    }
    return 0;
}

static void free_lists(olists *L) {
    free(L->rec);
    free(L->rects);
    free(L->status);
    free(L->off);
    free(L->ent);
}

/* Public: the tile lists of one camera. Call with ent_g == NULL to get the
 * number of entries; then with buffers of that size. off[ntiles+1] receives
 * the list offsets; ent_g / ent_flags (bit0 member, bit1 ambiguous membership,
 * bit2 depth within the band of the next entry) the entries in (z, index)
 * order; ent_z the double depth. Returns the entry count (or -1 on failure). */
int64_t or_tile_lists(int64_t n, int deg, const double *mean, const double *log_scale,
                      const double *quat, const double *logit, const double *sh,
                      const double *viewmat, const double *intr, int W, int H,
                      const double *prm, const double *band, int64_t *off, int64_t *ent_g,
                      int32_t *ent_flags, double *ent_z) {
    oscene s = {mean, log_scale, quat, logit, sh, n, deg};
    ocam c;
    make_cam(viewmat, intr, W, H, prm, &c);
    olists L;
    if (build_lists(&s, &c, prm, band, &L) != 0) {
        free_lists(&L);
        return -1;
    }
    int64_t total = L.off[L.ntiles];
    if (ent_g) {
        for (int t = 0; t <= L.ntiles; ++t) off[t] = L.off[t];
        for (int64_t k = 0; k < total; ++k) {
            ent_g[k] = L.ent[k].g;
            ent_flags[k] = (L.ent[k].prim ? 1 : 0) | (L.ent[k].amb ? 2 : 0) |
                           (L.ent[k].zswap ? 4 : 0);
            ent_z[k] = L.ent[k].z;
        }
    }
    free_lists(&L);
    return total;
}

/* ------------------------------------------------------------- compositing */

typedef struct {
    double rgb[3], D, T;
} oleaf;

typedef struct {
    const double *rec;
    double px, py;
    const double *prm;
    double lna_band, t_band;
    int maxleaf;
    oleaf *leaves;
    int nleaf;
    int overflow;
    /* primary-walk bookkeeping */
    int n_amb;
    int n_eval, n_alpha;
    int count;
} owalk;

static void emit(owalk *w, double T, const double *C, double D) {
    if (w->nleaf >= w->maxleaf) {
        w->overflow = 1;
        return;
    }
    oleaf *L = &w->leaves[w->nleaf++];
    L->rgb[0] = C[0] + T * w->prm[P_BG0];
    L->rgb[1] = C[1] + T * w->prm[P_BG1];
    L->rgb[2] = C[2] + T * w->prm[P_BG2];
    L->D = D;
    L->T = T;
}

/* Front-to-back compositing of one pixel over the list E[k..n), starting from
 * transmittance T, colour C and depth D:
 *   power = -1/2 (A dx^2 + C dy^2) - B dx dy, alpha = min(amax, o e^power);
 *   alpha < amin: skip;  T' = T (1 - alpha);  T' < T_min: stop (not added);
 *   C += alpha T c, D += alpha T z, T = T'.
 * Decisions within a band are flipped in spawned walks while `flips` > 0.
 * `fdec` >= 0 flips decision fdec of entry k (0 order, 1 membership, 2 alpha
 * skip, 3 termination) and suppresses spawning for decisions <= fdec there. */
static void walk(owalk *w, const oent *E, int64_t n, int64_t k, double T, const double *Cin,
                 double D, int flips, int fdec) {
    double C[3] = {Cin[0], Cin[1], Cin[2]};
    const double *prm = w->prm;
    for (; k < n; ++k, fdec = -1) {
        const oent *e = &E[k];
        if (e->zswap && k + 1 < n && fdec < 0) {
            if (w->count) w->n_amb++;
            if (flips > 0) {
                int64_t m = n - k;
                oent *cp = (oent *)malloc(sizeof(oent) * (size_t)m);
                if (cp) {
                    memcpy(cp, E + k, sizeof(oent) * (size_t)m);
                    oent tmp = cp[0];
                    cp[0] = cp[1];
                    cp[1] = tmp;
                    cp[0].zswap = 0;
                    cp[1].zswap = 0;
                    int save = w->count;
                    w->count = 0;
                    walk(w, cp, m, 0, T, C, D, flips - 1, -1);
                    w->count = save;
                    free(cp);
                }
            }
        }
        int inc = e->prim;
        if (e->amb) {
            if (fdec == 1)
                inc = !inc;
            else if (fdec < 1) {
                if (w->count) w->n_amb++;
                if (flips > 0) {
                    int save = w->count;
                    w->count = 0;
                    walk(w, E, n, k, T, C, D, flips - 1, 1);
                    w->count = save;
                }
            }
        }
        if (!inc) continue;
        const double *r = w->rec + e->g * R_COUNT;
        double dx = w->px - r[R_U], dy = w->py - r[R_V];
        double power = -0.5 * (r[R_CA] * dx * dx + r[R_CC] * dy * dy) - r[R_CB] * dx * dy;
        double araw = r[R_O] * exp(power);
        if (w->count) w->n_eval++;
        int skip = araw < prm[P_AMIN];
        if (w->lna_band > 0.0 && r[R_O] > 0.0 &&
            fabs(log(r[R_O]) + power - log(prm[P_AMIN])) <= w->lna_band) {
            if (fdec == 2)
                skip = !skip;
            else if (fdec < 2) {
                if (w->count) w->n_amb++;
                if (flips > 0) {
                    int save = w->count;
                    w->count = 0;
                    walk(w, E, n, k, T, C, D, flips - 1, 2);
                    w->count = save;
                }
            }
        }
        if (skip) continue;
        if (w->count) w->n_alpha++;
        double alpha = araw < prm[P_AMAX] ? araw : prm[P_AMAX];
        double Tn = T * (1.0 - alpha);
        int stop = Tn < prm[P_TMIN];
        if (w->t_band > 0.0 && fabs(Tn - prm[P_TMIN]) <= w->t_band * prm[P_TMIN]) {
            if (fdec == 3)
                stop = !stop;
            else if (fdec < 3) {
                if (w->count) w->n_amb++;
                if (flips > 0) {
                    int save = w->count;
                    w->count = 0;
                    walk(w, E, n, k, T, C, D, flips - 1, 3);
                    w->count = save;
                }
            }
        }
        if (stop) {
            emit(w, T, C, D);
            return;
        }
        double wt = alpha * T;
        C[0] += wt * r[R_RED];
        C[1] += wt * r[R_GRN];
        C[2] += wt * r[R_BLU];
        D += wt * r[R_Z];
        T = Tn;
    }
    emit(w, T, C, D);
}

/* Public: render one camera.
 * mode 0: per-tile lists (sorted once per tile, shared by its pixels);
 * mode 1: brute force (each pixel gathers and sorts its own list from all
 *         Gaussians; meant for tiny scenes).
 * Outputs (row-major H x W): rgb[3 per pixel], depth, T, flags (bit0: the
 * primary walk met a near-threshold decision; bit1: more alternatives than
 * max leaves), n_eval (pairs whose power was evaluated), n_alpha (pairs with
 * alpha >= amin, the terminating one included). Alternative results of
 * flagged pixels go to leaf_pix / leaf_val (rgb, D, T) up to leaf_cap entries.
 * Returns the total number of alternative leaves (may exceed leaf_cap: call
 * again with more room) or -1 on allocation failure. */
int64_t or_render(int64_t n, int deg, const double *mean, const double *log_scale,
                  const double *quat, const double *logit, const double *sh,
                  const double *viewmat, const double *intr, int W, int H, const double *prm,
                  const double *band, int mode, double *rgb, double *depth, double *Tout,
                  int32_t *flags, int32_t *n_eval, int32_t *n_alpha, int64_t leaf_cap,
                  int32_t *leaf_pix, double *leaf_val) {
    oscene s = {mean, log_scale, quat, logit, sh, n, deg};
    ocam c;
    make_cam(viewmat, intr, W, H, prm, &c);
    olists L;
    if (build_lists(&s, &c, prm, band, &L) != 0) {
        free_lists(&L);
        return -1;
    }
    int maxflip = (int)band[B_MAXFLIP];
    int maxleaf = (int)band[B_MAXLEAF];
    if (maxleaf < 1) maxleaf = 1;
    int64_t nleaf_total = 0; /* shared; advanced atomically */
    int failed = 0;

#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < L.ntiles; ++t) {
        int tx = t % c.TX, ty = t / c.TX;
        oleaf *leaves = (oleaf *)malloc(sizeof(oleaf) * (size_t)maxleaf);
        oent *own = NULL;
        if (mode == 1) own = (oent *)malloc(sizeof(oent) * (size_t)(n > 0 ? n : 1));
        if (!leaves || (mode == 1 && !own)) {
#pragma omp atomic write
            failed = 1;
            free(leaves);
            free(own);
            continue;
        }
        for (int j = ty * c.tile; j < (ty + 1) * c.tile && j < H; ++j)
            for (int i = tx * c.tile; i < (tx + 1) * c.tile && i < W; ++i) {
                const oent *E;
                int64_t m;
                if (mode == 1) {
                    /* gather every Gaussian whose widened rect contains this
                     * pixel's tile, then sort this pixel's own list */
                    m = 0;
                    int ptx = i / c.tile, pty = j / c.tile;
                    for (int64_t g = 0; g < n; ++g) {
                        if (!(L.status[g] & ST_PROJ)) continue;
                        const int32_t *r0 = L.rects + g * 12, *e = L.rects + g * 12 + 4,
                                      *in = L.rects + g * 12 + 8;
                        if (!rect_has(e, ptx, pty)) continue;
                        int st = L.status[g];
                        oent *o = &own[m++];
                        o->g = g;
                        o->z = L.rec[g * R_COUNT + R_Z];
                        o->prim = (st & ST_VALID) && rect_has(r0, ptx, pty);
                        int certain = (st & ST_VALID) && !(st & ST_AMBIG) && rect_has(in, ptx, pty);
                        o->amb = (unsigned char)!certain;
                        o->zswap = 0;
                    }
                    qsort(own, (size_t)m, sizeof(oent), ent_cmp);
                    for (int64_t k = 0; k + 1 < m; ++k) {
                        double dz = fabs(own[k + 1].z - own[k].z);
                        if ((band[B_Z_ABS] > 0.0 || band[B_Z_REL] > 0.0) &&
                            dz <= band[B_Z_ABS] + band[B_Z_REL] * fabs(own[k].z))
                            own[k].zswap = 1;
                    }
                    E = own;
                } else {
                    E = L.ent + L.off[t];
                    m = L.off[t + 1] - L.off[t];
                }
                owalk w;
                memset(&w, 0, sizeof(w));
                w.rec = L.rec;
                w.px = i + 0.5;
                w.py = j + 0.5;
                w.prm = prm;
                w.lna_band = band[B_LNA];
                w.t_band = band[B_T_REL];
                w.maxleaf = maxleaf;
                w.leaves = leaves;
                w.count = 1;
                double C0[3] = {0.0, 0.0, 0.0};
                /* primary walk: double-precision decisions only */
                walk(&w, E, m, 0, 1.0, C0, 0.0, 0, -1);
                int64_t p = (int64_t)j * W + i;
                rgb[3 * p + 0] = leaves[0].rgb[0];
                rgb[3 * p + 1] = leaves[0].rgb[1];
                rgb[3 * p + 2] = leaves[0].rgb[2];
                depth[p] = leaves[0].D;
                Tout[p] = leaves[0].T;
                n_eval[p] = w.n_eval;
                n_alpha[p] = w.n_alpha;
                int fl = w.n_amb > 0 ? 1 : 0;
                if (w.n_amb > 0 && maxflip > 0) {
                    /* alternatives: walks that flip up to maxflip decisions */
                    w.nleaf = 0;
                    w.count = 0;
                    walk(&w, E, m, 0, 1.0, C0, 0.0, maxflip, -1);
                    if (w.overflow) fl |= 2;
                    int64_t base;
#pragma omp atomic capture
                    {
                        base = nleaf_total;
                        nleaf_total += w.nleaf;
                    }
                    for (int q = 0; q < w.nleaf; ++q) {
                        int64_t o = base + q;
                        if (o < leaf_cap) {
                            leaf_pix[o] = (int32_t)p;
                            leaf_val[5 * o + 0] = leaves[q].rgb[0];
                            leaf_val[5 * o + 1] = leaves[q].rgb[1];
                            leaf_val[5 * o + 2] = leaves[q].rgb[2];
                            leaf_val[5 * o + 3] = leaves[q].D;
                            leaf_val[5 * o + 4] = leaves[q].T;
                        }
                    }
                }
                flags[p] = fl;
            }
        free(leaves);
        free(own);
    }
    free_lists(&L);
    return failed ? -1 : nleaf_total;
}
