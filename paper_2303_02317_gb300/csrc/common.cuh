// common.cuh -- device-side definitions shared by the pricer kernels.
//
// Lattice parameters follow the paper's models:
//   binomial call   Sec. 2.1 and Fig. 1 (weights m(1-p) on G[i+1][j], m p on
//                   G[i+1][j+1]; node price S u^{2j-i})
//   trinomial call  Sec. 3 and its appendix (weights m p_d, m p_o, m p_u on
//                   G[i+1][j..j+2]; node price S u^{j-i})
//   BSM put         Sec. 4, explicit scheme bsmG (weights b, c, a on k-1, k, k+1)
//   binomial and trinomial puts: priced as the call of the mirrored lattice
//                   (make_params below), so every kernel sees a call
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/american.h"

namespace aop {

constexpr int kMaxDepth = 24;          // D&C recursion depth bound
constexpr int kExpBits = 7;            // 3 x 7-bit exponent tables cover 2^21
constexpr int kExpTab = 1 << kExpBits;

// Per-option lattice description, computed on the device from an aop_request.
struct Params {
    int32_t model;       // aop_model
    int32_t status;      // aop_status of the setup
    int32_t D;           // columns added per row: 1 (binomial) or 2
    int32_t nw;          // stencil width (2 or 3)
    int32_t o_min;       // offset of w[0]: 0 (calls) or -1 (BSM)
    int32_t mirror;      // 1: a binomial/trinomial put priced as the mirrored call
    int64_t T;
    double w[3];         // weights on offsets o_min .. o_min+nw-1
    double wsum;         // sum of the weights = symbol at theta = 0
    double logu;         // log of the price factor per column (calls), ds (BSM)
    double S, K;
    double xbase;        // calls: ln S - T logu;  BSM: ln(S/K) - T ds
    double out_scale;    // 1 for the calls, K for the put (price = K v)
    double dt;           // calendar time per row, expiry / T (years)
    // Exponential tilt of the call stencil: a call value never exceeds its
    // node price S u^k, which grows like e^{kappa x} along a row, so tilted
    // convolutions carry v(x) e^{-kappa x} (kept near the local scale of the
    // node prices) with the tilted weights w_j e^{kappa j}, normalised to
    // unit sum: wt_j = w_j e^{kappa j} / e^{tL}.
    double kappa;        // log growth of the node price per column (0: BSM)
    double wt[3];
    double wtsum;
    double tL;           // log of the tilted weights' sum
};
static_assert(sizeof(Params) % 8 == 0, "Params alignment");

// Largest column index of row `row` (calls) / half-width of BSM row n.
__host__ __device__ inline int64_t row_last(const Params &P, int64_t row) {
    return P.model == AOP_BSM_PUT ? (P.T - row) : (int64_t)P.D * row;
}

// Exponent index k' = k + T in [0, 2T] for the exercise value of a cell.
//   binomial call: k = 2j - i   trinomial call: k = j - i   BSM: k = spatial index
__host__ __device__ inline int64_t ex_index(const Params &P, int64_t row, int64_t col) {
    if (P.model == AOP_BINOMIAL_CALL) return 2 * col - row + P.T;
    if (P.model == AOP_TRINOMIAL_CALL) return col - row + P.T;
    return col + P.T;
}

// e^{xbase + k' logu} from three 7-bit tables: t3[c] * t2[b] * t1[a] with
// k' = a + 128 b + 16384 c, t3[c] = e^{xbase + 16384 c logu} (the base folded
// into the coarse table so that no factor overflows when the node price itself
// is representable: node prices reach e^{+-650} at T = 2^17 for sigma = 0.6 and
// three years), t2[b] = e^{128 b logu}, t1[a] = e^{a logu}.  Each entry is one
// exp, so the product is within a few ulp of the exact node price.
struct ExpTables {
    double t1[kExpTab], t2[kExpTab], t3[kExpTab];
};

__device__ inline double exp_from_tables(const ExpTables &E, int64_t kp) {
    int a = (int)(kp & (kExpTab - 1));
    int b = (int)((kp >> kExpBits) & (kExpTab - 1));
    int c = (int)(kp >> (2 * kExpBits));
    return E.t3[c] * E.t2[b] * E.t1[a];
}

// Exercise value of the cell whose exponent index is kp.
//   calls: S u^k - K ;  BSM (units of K): 1 - e^{s_k}
__device__ inline double exercise(const Params &P, const ExpTables &E, int64_t kp) {
    double x = exp_from_tables(E, kp);
    return P.model == AOP_BSM_PUT ? 1.0 - x : x - P.K;
}

// Build the exponent tables cooperatively (all threads of the block call it).
__device__ inline void build_exp_tables(const Params &P, ExpTables &E) {
    for (int t = threadIdx.x; t < 3 * kExpTab; t += blockDim.x) {
        int tab = t / kExpTab, n = t % kExpTab;
        double scale = (double)(1ll << (kExpBits * tab));
        if (tab == 0) E.t1[n] = exp((double)n * P.logu);
        else if (tab == 1) E.t2[n] = exp((double)n * scale * P.logu);
        else E.t3[n] = exp(P.xbase + (double)n * scale * P.logu);
    }
}

// Lattice parameter setup (hot-path step a1).  Formulas as in the paper; the
// trinomial Boyle form solves the two-moment system in closed form.
//
// Binomial and trinomial puts.  Dividing a put value by its node price
// S u^x turns the put recursion into a call recursion on the same lattice,
// mirrored in j: with j' = D i - j the cell holds C = G S / (S u^x) and
//   C[i][j'] = max(sum_t w'_t C[i+1][j'+t], K u^{x'} - S),  x' = -x,
// where w'_t is the put's weight on the child at mirrored offset t times that
// child's price ratio (u^{+1} for the up child, u^{-1} for the down child).
// That is the call with spot K, strike S, discount per step e^{-q dt} and
// yield r (put-call symmetry of the lattice; McDonald and Schroder 1998), so
// the recursion, its red/green divider (Cor. 2.7 applied to the mirrored call)
// and every kernel below are the call's; only the boundary is mirrored back
// (last green put column = D i - 1 - last red mirrored column).  The weights
// are built from the put's own probabilities, so the identity is exact for
// both trinomial forms.
__device__ inline Params make_params(const aop_request &q) {
    Params P;
    const bool mirror = (q.model == AOP_BINOMIAL_PUT || q.model == AOP_TRINOMIAL_PUT);
    P.model = mirror ? q.model - AOP_BINOMIAL_PUT : q.model;
    P.status = AOP_OK;
    P.T = q.T;
    P.S = mirror ? q.K : q.S0;
    P.K = mirror ? q.S0 : q.K;
    P.w[0] = P.w[1] = P.w[2] = 0.0;
    P.mirror = mirror ? 1 : 0;
    P.out_scale = 1.0;
    P.dt = (q.T >= 1) ? q.expiry / (double)q.T : 0.0;
    if (!(q.S0 > 0) || !(q.K > 0) || !(q.sigma > 0) || !(q.expiry > 0) || q.T < 1 ||
        q.T > AOP_MAX_T || q.model < 0 || q.model > AOP_TRINOMIAL_PUT) {
        P.status = AOP_EINVAL;
        P.D = 1; P.nw = 2; P.o_min = 0; P.wsum = 1; P.logu = 0; P.xbase = 0;
        P.model = AOP_BINOMIAL_CALL; P.mirror = 0;
        return P;
    }
    const double T = (double)q.T;
    if (P.model == AOP_BINOMIAL_CALL) {
        double dt = q.expiry / T;
        double logu = q.sigma * sqrt(dt);
        double u = exp(logu);
        double d = 1.0 / u;
        double p = (exp((q.r - q.q) * dt) - d) / (u - d);
        double m = exp(-q.r * dt);
        if (!(p >= 0.0 && p <= 1.0)) P.status = AOP_EUNSTABLE;
        P.D = 1; P.nw = 2; P.o_min = 0;
        if (mirror) {                 // mirrored offset 0 = up child, 1 = down child
            P.w[0] = m * p * u;
            P.w[1] = m * (1.0 - p) * d;
        } else {
            P.w[0] = m * (1.0 - p);
            P.w[1] = m * p;
        }
        P.logu = logu;
        P.xbase = log(P.S) - T * logu;
    } else if (P.model == AOP_TRINOMIAL_CALL) {
        double dt = q.expiry / T;
        double m = exp(-q.r * dt);
        double logu, u, pu, pd, po;
        if (q.tri_form == AOP_TRI_PAPER) {
            logu = q.sigma * sqrt(2.0 * dt);
            u = exp(logu);
            double su = exp(q.sigma * sqrt(dt / 2.0));
            double sd = 1.0 / su;
            double e = exp((q.r - q.q) * dt / 2.0);
            pu = (e - sd) / (su - sd); pu = pu * pu;
            pd = (su - e) / (su - sd); pd = pd * pd;
            po = 1.0 - pu - pd;
        } else {
            double lam = q.lambda > 0 ? q.lambda : sqrt(3.0);
            logu = lam * q.sigma * sqrt(dt);
            u = exp(logu);
            // first and second moment of the price relative, relative to 1
            double r1 = expm1((q.r - q.q) * dt);
            double r2 = expm1((2.0 * (q.r - q.q) + q.sigma * q.sigma) * dt);
            double a11 = u - 1.0, a12 = 1.0 / u - 1.0;
            double a21 = u * u - 1.0, a22 = 1.0 / (u * u) - 1.0;
            double det = a11 * a22 - a12 * a21;
            pu = (r1 * a22 - a12 * r2) / det;
            pd = (a11 * r2 - a21 * r1) / det;
            po = 1.0 - pu - pd;
        }
        if (!(pu >= 0 && pd >= 0 && po >= 0)) P.status = AOP_EUNSTABLE;
        P.D = 2; P.nw = 3; P.o_min = 0;
        if (mirror) {                 // mirrored offsets 0, 1, 2 = up, middle, down child
            P.w[0] = m * pu * u; P.w[1] = m * po; P.w[2] = m * pd / u;
        } else {
            P.w[0] = m * pd; P.w[1] = m * po; P.w[2] = m * pu;
        }
        P.logu = logu;
        P.xbase = log(P.S) - T * logu;
    } else {
        // Sec. 5's scheme; a dividend yield q enters the first-derivative
        // term only: v_tau = v_ss + (omega_q - 1) v_s - omega v with
        // omega_q = 2(r - q)/sigma^2 (q = 0 is the paper's scheme).
        double dtau = q.sigma * q.sigma * q.expiry / (2.0 * T);
        double omega = 2.0 * q.r / (q.sigma * q.sigma);
        double omega_q = 2.0 * (q.r - q.q) / (q.sigma * q.sigma);
        double ds = sqrt(3.0 * dtau);
        double al = dtau / (ds * ds);
        double be = (omega_q - 1.0) * dtau / (2.0 * ds);
        double a = al + be, b = al - be;
        double c = 1.0 - a - b - omega * dtau;
        if (!(a >= 0 && b >= 0 && c >= 0)) P.status = (P.status ? P.status : AOP_EUNSTABLE);
        P.D = 2; P.nw = 3; P.o_min = -1;
        P.w[0] = b; P.w[1] = c; P.w[2] = a;
        P.logu = ds;
        P.xbase = log(q.S0 / q.K) - T * ds;
        P.out_scale = q.K;
    }
    P.wsum = P.w[0] + P.w[1] + P.w[2];
    P.kappa = P.model == AOP_BINOMIAL_CALL ? 2.0 * P.logu : (P.model == AOP_TRINOMIAL_CALL ? P.logu : 0.0);
    double ts = 0.0;
    for (int j = 0; j < 3; j++) {
        P.wt[j] = P.w[j] * exp(P.kappa * j);
        ts += P.wt[j];
    }
    for (int j = 0; j < 3; j++) P.wt[j] /= ts;
    P.wtsum = P.wt[0] + P.wt[1] + P.wt[2];
    P.tL = log(ts);
    return P;
}

// ---------------------------------------------------------------- utilities
__host__ __device__ inline int ilog2_ceil(int64_t x) {
    int l = 0;
    while (((int64_t)1 << l) < x) l++;
    return l;
}

__device__ inline void set_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

}  // namespace aop
