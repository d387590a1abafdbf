/*
 * oracle.c -- plain, slow, obviously correct FP64 CPU reference for the
 * American option lattices of "Fast American Option Pricing using Nonlinear
 * Stencils" (arXiv 2303.02317).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only tests/, the smoke check and the CPU-baseline leg of
 * bench.py do.  It shares no code, header, table or constant generator with
 * the CUDA library.
 *
 * What it computes (the plain definition the fast method must reproduce):
 *
 *   BOPM call  (Fig. 1; Sec. 2.1; Def. 2.1)
 *     dt = E/T, u = e^{V sqrt(dt)}, d = 1/u, p = (e^{(R-Y)dt} - d)/(u - d),
 *     m = e^{-R dt}; weight m(1-p) on the down child G[i+1][j] and m p on the
 *     up child G[i+1][j+1] (the reading of Sec. 2.1 under which the identity
 *     s0/u + s1 u = e^{-Y dt} in the proof of Lemma 2.2 holds);
 *     G[T][j] = max(0, S u^{2j-T} - K);
 *     G[i][j] = max(m(1-p) G[i+1][j] + m p G[i+1][j+1], S u^{2j-i} - K).
 *
 *   TOPM call  (Sec. 3; appendix, trinomial model)
 *     weights m p_d, m p_o, m p_u on G[i+1][j], G[i+1][j+1], G[i+1][j+2],
 *     exercise S u^{j-i} - K, row i holds j in [0, 2i].
 *     form 1 (the paper's): u = e^{V sqrt(2 dt)},
 *       p_u = ((e^{(R-Y)dt/2} - u^{-1/2})/(u^{1/2} - u^{-1/2}))^2,
 *       p_d = ((u^{1/2} - e^{(R-Y)dt/2})/(u^{1/2} - u^{-1/2}))^2,
 *       p_o = 1 - p_u - p_d.
 *     form 0 (Boyle 1986): u = e^{lambda V sqrt(dt)}, probabilities matching
 *       the first two moments of the price relative:
 *       p_u + p_o + p_d = 1,
 *       p_u u + p_o + p_d/u = e^{(R-Y)dt},
 *       p_u u^2 + p_o + p_d/u^2 = e^{(2(R-Y)+V^2)dt}.
 *
 *   BOPM put, TOPM put  (the exercise value of a put, Sec. 2.1)
 *     the same lattices, weights and rows as the calls, with exercise value
 *     K - S u^{2j-i} (binomial) or K - S u^{j-i} (trinomial).
 *
 *   BSM put  (Sec. 4, explicit scheme bsmG)
 *     dtau = V^2 E/(2T), omega = 2R/V^2, ds = sqrt(3 dtau),
 *     a = dtau/ds^2 + (omega-1) dtau/(2 ds) on k+1,
 *     b = dtau/ds^2 - (omega-1) dtau/(2 ds) on k-1,
 *     c = 1 - a - b - omega dtau on k,
 *     s_k = ln(S/K) + k ds, v^0_k = max(1 - e^{s_k}, 0),
 *     v^{n+1}_k = max(a v^n_{k+1} + c v^n_k + b v^n_{k-1}, 1 - e^{s_k})
 *     on the shrinking triangle |k| <= T-n-1; price = K v^T_0.
 *     With a dividend yield Y (absent from the paper, whose Sec. 4 sets none):
 *     the substitution that yields Sec. 5's nondimensional equation gives
 *     v_tau = v_ss + (omega_Y - 1) v_s - omega v with omega_Y = 2(R-Y)/V^2,
 *     so omega_Y replaces omega in the first-derivative term of a and b while
 *     omega stays in c; Y = 0 is the paper's scheme unchanged.
 *
 * Boundary outputs (Cor. 2.7 and the BSM boundary theorem):
 *   call: boundary[i] = largest j in [0, D i] whose continuation value is >=
 *         its exercise value (row T: continuation 0), -1 if none.
 *   BOPM/TOPM put: boundary[i] = largest j in [0, D i] whose exercise value
 *         is > its continuation value (row T: continuation 0), -1 if none.
 *   BSM put: boundary[n] = largest k in [-(T-n), T-n] whose exercise value is >
 *         its continuation value (row 0: continuation 0), INT32_MIN if none.
 *   margin[row] (optional) = min |continuation - exercise| over the divider
 *         cell and its right neighbour in that row (in price units for the
 *         lattices, in units of K for the BSM put); it measures how close a row
 *         is to a tie.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_BOPM = 0, OR_TOPM = 1, OR_BSM = 2, OR_BOPM_PUT = 3, OR_TOPM_PUT = 4 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_EUNSTABLE = 2, OR_ENOMEM = 3 };

typedef struct {
    int32_t model;
    int32_t tri_form;   /* TOPM: 0 = Boyle moment matching, 1 = paper form */
    double S, K, R, Y, V, E;   /* paper notation: spot, strike, rate, yield, vol, expiry (years) */
    int64_t T;
    double lambda;      /* TOPM form 0 stretch; <= 0 selects sqrt(3) */
} or_req;

typedef struct {
    int32_t model;
    int32_t D;          /* columns added per row: 1 BOPM, 2 TOPM, 2 BSM (2T+1 points) */
    double w[3];        /* stencil weights on offsets o_min .. o_min+2 */
    int32_t o_min;      /* 0 for the calls, -1 for BSM */
    int32_t nw;         /* 2 or 3 */
    double u;           /* price factor per column (calls) or e^{ds} (BSM) */
    double logu;        /* exact log of u as defined (V sqrt(dt), ...) */
    double dt, dtau, ds, omega, p, pu, po, pd, m;
    double omega_y;     /* BSM: 2(R-Y)/V^2, the drift coefficient */
} or_params;

static int is_lattice_put(int model) { return model == OR_BOPM_PUT || model == OR_TOPM_PUT; }

int or_params_compute(const or_req *q, or_params *P)
{
    memset(P, 0, sizeof(*P));
    if (!(q->S > 0) || !(q->K > 0) || !(q->V > 0) || !(q->E > 0) || q->T < 1)
        return OR_EINVAL;
    P->model = q->model;
    const double T = (double)q->T;
    if (q->model == OR_BOPM || q->model == OR_BOPM_PUT) {
        double dt = q->E / T;
        double u = exp(q->V * sqrt(dt));
        double d = 1.0 / u;
        double p = (exp((q->R - q->Y) * dt) - d) / (u - d);
        double m = exp(-q->R * dt);
        if (!(p >= 0.0 && p <= 1.0)) return OR_EUNSTABLE;
        P->D = 1; P->nw = 2; P->o_min = 0;
        P->w[0] = m * (1.0 - p);   /* down child G[i+1][j]  */
        P->w[1] = m * p;           /* up child   G[i+1][j+1] */
        P->u = u; P->logu = q->V * sqrt(dt); P->dt = dt; P->p = p; P->m = m;
        return OR_OK;
    }
    if (q->model == OR_TOPM || q->model == OR_TOPM_PUT) {
        double dt = q->E / T;
        double m = exp(-q->R * dt);
        double u, logu, pu, pd, po;
        if (q->tri_form == 1) {
            logu = q->V * sqrt(2.0 * dt);
            u = exp(logu);
            double su = exp(q->V * sqrt(dt / 2.0));
            double sd = 1.0 / su;
            double e = exp((q->R - q->Y) * dt / 2.0);
            pu = (e - sd) / (su - sd); pu = pu * pu;
            pd = (su - e) / (su - sd); pd = pd * pd;
            po = 1.0 - pu - pd;
        } else {
            double lam = q->lambda > 0 ? q->lambda : sqrt(3.0);
            logu = lam * q->V * sqrt(dt);
            u = exp(logu);
            /* Solve the 3x3 moment system by Gaussian elimination on the
               unknowns (pu, po, pd); rows: sum, first moment, second moment.
               Right-hand sides are taken relative to 1 (expm1) so that the
               O(dt) quantities keep full precision. */
            double r1 = expm1((q->R - q->Y) * dt);
            double r2 = expm1((2.0 * (q->R - q->Y) + q->V * q->V) * dt);
            /* subtract row 0 from rows 1 and 2: po drops out */
            double a11 = u - 1.0,       a12 = 1.0 / u - 1.0;
            double a21 = u * u - 1.0,   a22 = 1.0 / (u * u) - 1.0;
            double det = a11 * a22 - a12 * a21;
            pu = (r1 * a22 - a12 * r2) / det;
            pd = (a11 * r2 - a21 * r1) / det;
            po = 1.0 - pu - pd;
        }
        if (!(pu >= 0 && pd >= 0 && po >= 0)) return OR_EUNSTABLE;
        P->D = 2; P->nw = 3; P->o_min = 0;
        P->w[0] = m * pd; P->w[1] = m * po; P->w[2] = m * pu;
        P->u = u; P->logu = logu; P->dt = dt; P->pu = pu; P->po = po; P->pd = pd; P->m = m;
        return OR_OK;
    }
    if (q->model == OR_BSM) {
        double dtau = q->V * q->V * q->E / (2.0 * T);
        double omega = 2.0 * q->R / (q->V * q->V);
        double omega_y = 2.0 * (q->R - q->Y) / (q->V * q->V);
        double ds = sqrt(3.0 * dtau);
        double al = dtau / (ds * ds);
        double be = (omega_y - 1.0) * dtau / (2.0 * ds);
        double a = al + be, b = al - be;
        double c = 1.0 - a - b - omega * dtau;
        if (!(a >= 0 && b >= 0 && c >= 0)) return OR_EUNSTABLE;
        P->D = 2; P->nw = 3; P->o_min = -1;
        P->w[0] = b; P->w[1] = c; P->w[2] = a;   /* on k-1, k, k+1 */
        P->u = exp(ds); P->logu = ds; P->dtau = dtau; P->ds = ds; P->omega = omega;
        P->omega_y = omega_y;
        return OR_OK;
    }
    return OR_EINVAL;
}

/* exercise value table ex[k + T] for k in [-T, T]:
   calls: S u^k - K with u^k evaluated as e^{k log u} from the exact log u of
   the model (Sec. 2.1: node price S u^{N_u - N_d}); lattice puts: K - S u^k;
   BSM put: 1 - e^{ln(S/K) + k ds} (units of K). */
static double *exercise_table(const or_req *q, const or_params *P)
{
    int64_t T = q->T;
    double *ex = (double *)malloc(sizeof(double) * (size_t)(2 * T + 1));
    if (!ex) return NULL;
    for (int64_t k = -T; k <= T; k++) {
        if (P->model == OR_BSM)
            ex[k + T] = 1.0 - exp(log(q->S / q->K) + (double)k * P->ds);
        else if (is_lattice_put(P->model))
            ex[k + T] = q->K - q->S * exp((double)k * P->logu);
        else
            ex[k + T] = q->S * exp((double)k * P->logu) - q->K;
    }
    return ex;
}

/*
 * Core backward induction.  american = 0 drops the max (European value on the
 * same lattice).  grid (optional) receives every row: row r of the call grid is
 * at grid[r*(D*T+1) + j]; row n of the put grid at grid[n*(2T+1) + (k+T)].
 * near (optional, 8 doubles) receives the rows next to the root: lattices:
 * row 1 (j = 0..D) at near[0..], row 2 (j = 0..2D) at near[3..]; BSM: row
 * T-1 (k = -1..1) at near[0..2], row T-2 (k = -2..2) at near[3..7].
 */
static int lattice(const or_req *q, int american, int nthreads, double *price,
                   int32_t *boundary, double *margin, double *grid, double *near)
{
    or_params P;
    int st = or_params_compute(q, &P);
    if (st) return st;
    const int64_t T = q->T;
    const int64_t W = (P.model == OR_BSM) ? 2 * T + 1 : P.D * T + 1;
    double *ex = exercise_table(q, &P);
    double *cur = (double *)malloc(sizeof(double) * (size_t)W);
    double *nxt = (double *)malloc(sizeof(double) * (size_t)W);
    if (!ex || !cur || !nxt) { free(ex); free(cur); free(nxt); return OR_ENOMEM; }
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    (void)nthreads;
#endif

    if (P.model != OR_BSM) {
        const int D = P.D;
        const int put = is_lattice_put(P.model);
        const double w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
        /* leaves, row T: continuation 0.  The divider is the last red cell
           (call) or the last green cell (put). */
        int64_t last = -1;
        for (int64_t j = 0; j <= D * T; j++) {
            int64_t k = (D == 1) ? 2 * j - T : j - T;
            double e = ex[k + T];
            cur[j] = e > 0.0 ? e : 0.0;
            if (put ? (e > 0.0) : (0.0 >= e)) last = j;
        }
        if (boundary) boundary[T] = (int32_t)last;
        if (margin) {
            double mg = INFINITY;
            if (last >= 0) mg = fmin(mg, fabs(0.0 - ex[((D == 1) ? 2 * last - T : last - T) + T]));
            if (last + 1 <= D * T) mg = fmin(mg, fabs(0.0 - ex[((D == 1) ? 2 * (last + 1) - T : last + 1 - T) + T]));
            margin[T] = mg;
        }
        if (grid) memcpy(grid + (size_t)T * W, cur, sizeof(double) * (size_t)W);
        for (int64_t i = T - 1; i >= 0; i--) {
            const int64_t n = D * i;   /* last column of row i */
            #pragma omp parallel for num_threads(nthreads) schedule(static) if (n > 4096)
            for (int64_t j = 0; j <= n; j++) {
                double cont = (D == 1) ? w0 * cur[j] + w1 * cur[j + 1]
                                       : w0 * cur[j] + w1 * cur[j + 1] + w2 * cur[j + 2];
                int64_t k = (D == 1) ? 2 * j - i : j - i;
                double e = ex[k + T];
                nxt[j] = (american && e > cont) ? e : cont;
            }
            if (boundary || margin) {
                /* largest j with continuation >= exercise (call) or with
                   exercise > continuation (put), found by rescanning */
                int64_t br = -1;
                for (int64_t j = n; j >= 0; j--) {
                    double cont = (D == 1) ? w0 * cur[j] + w1 * cur[j + 1]
                                           : w0 * cur[j] + w1 * cur[j + 1] + w2 * cur[j + 2];
                    int64_t k = (D == 1) ? 2 * j - i : j - i;
                    if (put ? (ex[k + T] > cont) : (cont >= ex[k + T])) { br = j; break; }
                }
                if (boundary) boundary[i] = (int32_t)br;
                if (margin) {
                    double mg = INFINITY;
                    for (int64_t j = br; j <= br + 1; j++) {
                        if (j < 0 || j > n) continue;
                        double cont = (D == 1) ? w0 * cur[j] + w1 * cur[j + 1]
                                               : w0 * cur[j] + w1 * cur[j + 1] + w2 * cur[j + 2];
                        int64_t k = (D == 1) ? 2 * j - i : j - i;
                        mg = fmin(mg, fabs(cont - ex[k + T]));
                    }
                    margin[i] = mg;
                }
            }
            double *t = cur; cur = nxt; nxt = t;
            if (near && i == 1) for (int j = 0; j <= D; j++) near[j] = cur[j];
            if (near && i == 2) for (int j = 0; j <= 2 * D; j++) near[3 + j] = cur[j];
            if (grid) {
                memcpy(grid + (size_t)i * W, cur, sizeof(double) * (size_t)(n + 1));
                for (int64_t j = n + 1; j < W; j++) grid[(size_t)i * W + j] = NAN;
            }
        }
        *price = cur[0];
    } else {
        const double b = P.w[0], c = P.w[1], a = P.w[2];
        /* row 0 on k in [-T, T], stored at index k + T */
        int64_t last_green = INT64_MIN;
        for (int64_t k = -T; k <= T; k++) {
            double e = ex[k + T];
            cur[k + T] = e > 0.0 ? e : 0.0;
            if (e > 0.0) last_green = k;
        }
        if (boundary) boundary[0] = last_green == INT64_MIN ? INT32_MIN : (int32_t)last_green;
        if (margin) {
            double mg = INFINITY;
            int64_t lg = last_green == INT64_MIN ? -T - 1 : last_green;
            for (int64_t k = lg; k <= lg + 1; k++)
                if (k >= -T && k <= T) mg = fmin(mg, fabs(ex[k + T] - 0.0));
            margin[0] = mg;
        }
        if (grid) memcpy(grid, cur, sizeof(double) * (size_t)W);
        for (int64_t n = 1; n <= T; n++) {
            const int64_t R = T - n;   /* row n spans k in [-R, R] */
            #pragma omp parallel for num_threads(nthreads) schedule(static) if (R > 2048)
            for (int64_t k = -R; k <= R; k++) {
                double cont = b * cur[k - 1 + T] + c * cur[k + T] + a * cur[k + 1 + T];
                double e = ex[k + T];
                nxt[k + T] = (american && e > cont) ? e : cont;
            }
            if (boundary || margin) {
                int64_t bg = INT64_MIN;
                for (int64_t k = R; k >= -R; k--) {
                    double cont = b * cur[k - 1 + T] + c * cur[k + T] + a * cur[k + 1 + T];
                    if (ex[k + T] > cont) { bg = k; break; }
                }
                if (boundary) boundary[n] = bg == INT64_MIN ? INT32_MIN : (int32_t)bg;
                if (margin) {
                    double mg = INFINITY;
                    int64_t lg = bg == INT64_MIN ? -R - 1 : bg;
                    for (int64_t k = lg; k <= lg + 1; k++) {
                        if (k < -R || k > R) continue;
                        double cont = b * cur[k - 1 + T] + c * cur[k + T] + a * cur[k + 1 + T];
                        mg = fmin(mg, fabs(ex[k + T] - cont));
                    }
                    margin[n] = mg;
                }
            }
            double *t = cur; cur = nxt; nxt = t;
            if (near && n == T - 1) for (int k = -1; k <= 1; k++) near[k + 1] = cur[k + T];
            if (near && n == T - 2) for (int k = -2; k <= 2; k++) near[k + 5] = cur[k + T];
            /* cells outside [-R, R] keep stale values; they are never read again */
            if (grid) {
                for (int64_t k = -T; k <= T; k++)
                    grid[(size_t)n * W + (k + T)] = (k >= -R && k <= R) ? cur[k + T] : NAN;
            }
        }
        *price = q->K * cur[T];
    }
    free(ex); free(cur); free(nxt);
    return OR_OK;
}

int or_price_american(const or_req *q, int nthreads, double *price, int32_t *boundary, double *margin)
{
    return lattice(q, 1, nthreads, price, boundary, margin, NULL, NULL);
}

int or_price_european(const or_req *q, int nthreads, double *price)
{
    return lattice(q, 0, nthreads, price, NULL, NULL, NULL, NULL);
}

/*
 * Sensitivities from the nodes next to the root (textbook lattice estimates,
 * e.g. Hull, "Options, Futures and Other Derivatives", binomial trees):
 *   binomial:  delta = (G[1][1] - G[1][0]) / (S u - S d)
 *              gamma = ((G[2][2] - G[2][1]) / (S u^2 - S) - (G[2][1] - G[2][0]) / (S - S d^2))
 *                      / ((S u^2 - S d^2) / 2)
 *              theta = (G[2][1] - G[0][0]) / (2 dt)
 *   trinomial: the same differences on row 1 (spots S d, S, S u),
 *              theta = (G[1][1] - G[0][0]) / dt
 *   BSM put:   the same on row T-1 (spots S e^{-ds}, S, S e^{ds}), values K v,
 *              theta = K (v^{T-1}_0 - v^T_0) / dt
 * with dt = E/T and node spots S e^{x log u}.  out = {price, delta, gamma,
 * theta}; near (optional, 8 doubles) as in lattice().  Needs T >= 3.
 */
int or_greeks(const or_req *q, int american, int nthreads, double *out, double *near_out)
{
    if (q->T < 3) return OR_EINVAL;
    or_params P;
    int st = or_params_compute(q, &P);
    if (st) return st;
    double near[8], price;
    st = lattice(q, american, nthreads, &price, NULL, NULL, NULL, near);
    if (st) return st;
    const double S = q->S, dt = q->E / (double)q->T;
    double delta, gamma, theta;
    if (P.model == OR_BSM) {
        const double su = S * exp(P.ds), s0 = S, sd = S * exp(-P.ds);
        const double vd = q->K * near[0], v0 = q->K * near[1], vu = q->K * near[2];
        delta = (vu - vd) / (su - sd);
        gamma = ((vu - v0) / (su - s0) - (v0 - vd) / (s0 - sd)) / ((su - sd) / 2.0);
        theta = (v0 - price) / dt;
    } else if (P.D == 1) {
        const double s1u = S * exp(P.logu), s1d = S * exp(-P.logu);
        const double s2u = S * exp(2.0 * P.logu), s2d = S * exp(-2.0 * P.logu);
        delta = (near[1] - near[0]) / (s1u - s1d);
        gamma = ((near[5] - near[4]) / (s2u - S) - (near[4] - near[3]) / (S - s2d)) / ((s2u - s2d) / 2.0);
        theta = (near[4] - price) / (2.0 * dt);
    } else {
        const double s1u = S * exp(P.logu), s1d = S * exp(-P.logu);
        delta = (near[2] - near[0]) / (s1u - s1d);
        gamma = ((near[2] - near[1]) / (s1u - S) - (near[1] - near[0]) / (S - s1d)) / ((s1u - s1d) / 2.0);
        theta = (near[1] - price) / dt;
    }
    out[0] = price; out[1] = delta; out[2] = gamma; out[3] = theta;
    if (near_out) memcpy(near_out, near, sizeof(near));
    return OR_OK;
}

/* Full grid for small T (tests of the structural lemmas). */
int or_grid(const or_req *q, int american, double *grid, int32_t *boundary)
{
    double price;
    return lattice(q, american, 1, &price, boundary, NULL, grid, NULL);
}

/* Price many options one after another (the timed CPU baseline). */
int or_price_many(int64_t n, const or_req *qs, int nthreads, double *prices, int32_t *status)
{
    int bad = 0;
    for (int64_t i = 0; i < n; i++) {
        int st = or_price_american(&qs[i], nthreads, &prices[i], NULL, NULL);
        if (status) status[i] = st;
        if (st) { prices[i] = NAN; bad = 1; }
    }
    return bad ? OR_EINVAL : OR_OK;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int or_sizeof_req(void) { return (int)sizeof(or_req); }
