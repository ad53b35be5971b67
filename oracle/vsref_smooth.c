/*
 * vsref_smooth.c -- plain, slow CPU oracle for the temperature-smoothed
 * (log-domain sum-product) variant of the belief propagation of Eq. 1 in
 * "Towards Real-time 3D Reconstruction using Consumer UAVs" (arXiv 1902.09733),
 * and its reverse-mode derivative.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may build, load or call it.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * The paper's messages (Eq. 1) are min-sum: M(d) = min_d' [h(d') + V(d, d')].
 * Replacing the minimum by the soft minimum at temperature tau,
 *     softmin_tau(x) = -tau * log sum exp(-x / tau),
 * gives the log-domain sum-product message used here; as tau -> 0 it returns
 * to the min-sum message.  Everything is double precision, every message is
 * written out from this definition (O(L^2) per message, no factoring), and
 * the derivative is the plain chain rule taken step by step backwards through
 * the same loops, with every iteration's messages stored.
 *
 * Model (the same grid, directions and borders as the min-sum path):
 *   D[y][x][d]               data term, L labels, any real values
 *   V(d, d') = lam*|d-d'| if that is below T, else T     (truncated linear)
 *   slot k of pixel p holds the message from its neighbour p + off(k),
 *   off = {(-1,0), (+1,0), (0,-1), (0,+1)} (left, right, up, down);
 *   a neighbour outside the frame sends nothing: its slot stays 0.
 *   Schedule: synchronous.  Iteration t computes every message from the
 *   messages of iteration t-1 (all zero at t = 0):
 *     h(d')      = D_p(d') + sum over the other in-frame slots j != k of m_j(d')
 *     mt(d)      = -tau * log sum_d' exp(-(h(d') + V(d, d')) / tau)
 *     m_{p->q}   = mt - mean_d mt                        (mean normalisation)
 *   written to slot k^1 of q = p + off(k).
 *   Beliefs after the last iteration: b_p(d) = D_p(d) + sum_j m_j(d).
 *
 * Status codes: 0 ok, -1 invalid argument.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define SPREF_OK 0
#define SPREF_EINVAL (-1)

static const int OFF_X[4] = {-1, 1, 0, 0};
static const int OFF_Y[4] = {0, 0, -1, 1};

/* Truncated linear pairwise term and its partial derivatives in lam and T
 * (one-sided at the kink lam*|d-d'| == T, where V takes the T branch). */
static double v_term(int d, int dd, double lam, double T)
{
    double x = lam * (double)abs(d - dd);
    return x < T ? x : T;
}

static double v_dlam(int d, int dd, double lam, double T)
{
    double x = lam * (double)abs(d - dd);
    return x < T ? (double)abs(d - dd) : 0.0;
}

static double v_dT(int d, int dd, double lam, double T)
{
    double x = lam * (double)abs(d - dd);
    return x < T ? 0.0 : 1.0;
}

static int in_frame(int x, int y, int W, int H)
{
    return x >= 0 && y >= 0 && x < W && y < H;
}

/*
 * One smoothed message from the vector h (L values):
 *   mt(d) = -tau log sum_d' exp(-(h(d') + V(d,d'))/tau), evaluated with the
 *   minimum over d' of the exponent subtracted first (exact rewrite);
 * out = mt - mean(mt).  mt_out (nullable) receives mt before normalisation.
 */
void vsref_sp_message(const double *h, int L, double lam, double T, double tau,
                      double *out, double *mt_out)
{
    double *mt = (double *)malloc(sizeof(double) * (size_t)L);
    double mean = 0.0;
    for (int d = 0; d < L; ++d) {
        double mn = INFINITY;
        for (int dd = 0; dd < L; ++dd) {
            double e = h[dd] + v_term(d, dd, lam, T);
            if (e < mn)
                mn = e;
        }
        double z = 0.0;
        for (int dd = 0; dd < L; ++dd)
            z += exp(-(h[dd] + v_term(d, dd, lam, T) - mn) / tau);
        mt[d] = mn - tau * log(z);
        mean += mt[d];
    }
    mean /= (double)L;
    for (int d = 0; d < L; ++d) {
        out[d] = mt[d] - mean;
        if (mt_out)
            mt_out[d] = mt[d];
    }
    free(mt);
}

/* h(d') for the message that pixel (x, y) sends through slot direction k,
 * from the message state m ([4][H][W][L]). */
static void gather_h(const double *D, const double *m, int W, int H, int L,
                     int x, int y, int k, double *h)
{
    size_t p = (size_t)y * W + x;
    size_t plane = (size_t)W * H * L;
    for (int d = 0; d < L; ++d)
        h[d] = D[p * L + d];
    for (int j = 0; j < 4; ++j) {
        if (j == k || !in_frame(x + OFF_X[j], y + OFF_Y[j], W, H))
            continue;
        for (int d = 0; d < L; ++d)
            h[d] += m[j * plane + p * L + d];
    }
}

/*
 * Forward pass.  D: [H][W][L].  states: (iters + 1) message states of
 * [4][H][W][L] doubles each; state 0 is written as zeros.  beliefs: [H][W][L].
 */
int vsref_sp_forward(const double *D, int W, int H, int L, int iters,
                     double lam, double T, double tau, double *states, double *beliefs)
{
    if (W < 1 || H < 1 || L < 2 || iters < 0 || !(tau > 0.0) || lam < 0.0 || T < 0.0)
        return SPREF_EINVAL;
    size_t plane = (size_t)W * H * L;
    size_t state = 4 * plane;
    double *h = (double *)malloc(sizeof(double) * (size_t)L);
    double *out = (double *)malloc(sizeof(double) * (size_t)L);
    memset(states, 0, sizeof(double) * state);
    for (int t = 1; t <= iters; ++t) {
        const double *prev = states + (size_t)(t - 1) * state;
        double *cur = states + (size_t)t * state;
        memset(cur, 0, sizeof(double) * state);
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int k = 0; k < 4; ++k) {
                    int qx = x + OFF_X[k], qy = y + OFF_Y[k];
                    if (!in_frame(qx, qy, W, H))
                        continue;
                    gather_h(D, prev, W, H, L, x, y, k, h);
                    vsref_sp_message(h, L, lam, T, tau, out, NULL);
                    size_t q = (size_t)qy * W + qx;
                    /* q receives it in the slot facing p: k ^ 1 */
                    memcpy(cur + (size_t)(k ^ 1) * plane + q * L, out, sizeof(double) * (size_t)L);
                }
    }
    const double *last = states + (size_t)iters * state;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            for (int d = 0; d < L; ++d) {
                double b = D[p * L + d];
                for (int j = 0; j < 4; ++j)
                    if (in_frame(x + OFF_X[j], y + OFF_Y[j], W, H))
                        b += last[j * plane + p * L + d];
                beliefs[p * L + d] = b;
            }
        }
    free(h);
    free(out);
    return SPREF_OK;
}

/*
 * Reverse pass.  Given gbel = dLoss/dbeliefs ([H][W][L]) and the states of the
 * forward pass with the same arguments, writes gD = dLoss/dD ([H][W][L]) and
 * gpar = {dLoss/dlam, dLoss/dT, dLoss/dtau}.
 *
 * For one message with weights w(d,d') = exp(-(E(d,d') - mt(d))/tau),
 * E = h(d') + V(d,d') (each row of w sums to 1), and gt = g - mean(g) the
 * gradient passed through the mean normalisation:
 *   dLoss/dh(d')  = sum_d gt(d) w(d,d')
 *   dLoss/dlam   += sum_d gt(d) sum_d' w(d,d') dV/dlam
 *   dLoss/dT     += sum_d gt(d) sum_d' w(d,d') dV/dT
 *   dLoss/dtau   += sum_d gt(d) (mt(d) - sum_d' w(d,d') E(d,d')) / tau
 * (the last from differentiating -tau log sum exp(-E/tau) in tau).
 */
int vsref_sp_backward(const double *D, int W, int H, int L, int iters,
                      double lam, double T, double tau, const double *states,
                      const double *gbel, double *gD, double *gpar)
{
    if (W < 1 || H < 1 || L < 2 || iters < 0 || !(tau > 0.0) || lam < 0.0 || T < 0.0)
        return SPREF_EINVAL;
    size_t plane = (size_t)W * H * L;
    size_t state = 4 * plane;
    double *gm = (double *)calloc(state, sizeof(double));   /* adjoint of state t   */
    double *gp = (double *)calloc(state, sizeof(double));   /* adjoint of state t-1 */
    double *h = (double *)malloc(sizeof(double) * (size_t)L);
    double *gt = (double *)malloc(sizeof(double) * (size_t)L);
    double *hb = (double *)malloc(sizeof(double) * (size_t)L);
    double *mt = (double *)malloc(sizeof(double) * (size_t)L);
    double *wrow = (double *)malloc(sizeof(double) * (size_t)L);
    double glam = 0.0, gT = 0.0, gtau = 0.0;

    /* beliefs: b_p = D_p + sum of the in-frame slots of the last state */
    memcpy(gD, gbel, sizeof(double) * plane);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            for (int j = 0; j < 4; ++j)
                if (in_frame(x + OFF_X[j], y + OFF_Y[j], W, H))
                    memcpy(gm + j * plane + p * L, gbel + p * L, sizeof(double) * (size_t)L);
        }

    for (int t = iters; t >= 1; --t) {
        const double *prev = states + (size_t)(t - 1) * state;
        memset(gp, 0, sizeof(double) * state);
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int k = 0; k < 4; ++k) {
                    int qx = x + OFF_X[k], qy = y + OFF_Y[k];
                    if (!in_frame(qx, qy, W, H))
                        continue;
                    size_t p = (size_t)y * W + x;
                    size_t q = (size_t)qy * W + qx;
                    gather_h(D, prev, W, H, L, x, y, k, h);
                    /* the gradient of the message p -> q, through the normalisation */
                    const double *g = gm + (size_t)(k ^ 1) * plane + q * L;
                    double gmean = 0.0;
                    for (int d = 0; d < L; ++d)
                        gmean += g[d];
                    gmean /= (double)L;
                    for (int d = 0; d < L; ++d)
                        gt[d] = g[d] - gmean;
                    for (int d = 0; d < L; ++d)
                        hb[d] = 0.0;
                    for (int d = 0; d < L; ++d) {
                        /* row d of the soft-min: shift, partition sum, weights */
                        double mn = INFINITY;
                        for (int dd = 0; dd < L; ++dd) {
                            double e = h[dd] + v_term(d, dd, lam, T);
                            if (e < mn)
                                mn = e;
                        }
                        double z = 0.0;
                        for (int dd = 0; dd < L; ++dd) {
                            wrow[dd] = exp(-(h[dd] + v_term(d, dd, lam, T) - mn) / tau);
                            z += wrow[dd];
                        }
                        mt[d] = mn - tau * log(z);
                        double ew = 0.0, wl = 0.0, wT = 0.0;
                        for (int dd = 0; dd < L; ++dd) {
                            wrow[dd] /= z;
                            hb[dd] += gt[d] * wrow[dd];
                            wl += wrow[dd] * v_dlam(d, dd, lam, T);
                            wT += wrow[dd] * v_dT(d, dd, lam, T);
                            ew += wrow[dd] * (h[dd] + v_term(d, dd, lam, T));
                        }
                        glam += gt[d] * wl;
                        gT += gt[d] * wT;
                        gtau += gt[d] * (mt[d] - ew) / tau;
                    }
                    /* h = D_p + the other in-frame slots of p */
                    for (int d = 0; d < L; ++d)
                        gD[p * L + d] += hb[d];
                    for (int j = 0; j < 4; ++j) {
                        if (j == k || !in_frame(x + OFF_X[j], y + OFF_Y[j], W, H))
                            continue;
                        for (int d = 0; d < L; ++d)
                            gp[j * plane + p * L + d] += hb[d];
                    }
                }
        double *sw = gm;
        gm = gp;
        gp = sw;
    }
    gpar[0] = glam;
    gpar[1] = gT;
    gpar[2] = gtau;
    free(gm);
    free(gp);
    free(h);
    free(gt);
    free(hb);
    free(mt);
    free(wrow);
    return SPREF_OK;
}
