/*
 * The joint Kalman filter of a pulsar timing array with a stochastic
 * gravitational-wave background (GWB) whose per-pulsar redshifts are coupled
 * by the Hellings-Downs correlation, written once for a scalar type KF_T and
 * included twice by gwb.c (double, and double complex for complex-step
 * derivatives).
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle.
 *
 * Model (paper, Functionality: OU red noise and the GWB as linear SDEs
 * compiled into one state-space model, Hellings-Downs correlations in the
 * covariance that couples the processes across pulsars; corner-plot
 * parameters h_a, gamma_a, sigma_p, gamma_p, EFAC, EQUAD).  Per pulsar n the
 * state is (rho_n, y_n, a_n):
 *   d rho_n = (y_n + a_n) dt,
 *   d y_n   = -gamma_p,n y_n dt + sigma_p,n dW_n        (independent),
 *   d a_n   = -gamma_a a_n dt + h_a dB_n,  <dB_n dB_m> = G_nm dt  (HD),
 *   r_k = rho_{n_k}(t_k) + eps_k,  eps_k ~ N(0, EFAC^2 sigma_k^2 + EQUAD^2).
 * At the array's earliest TOA t_0: (rho_n, y_n) ~ N(0, P0_n), independent;
 * a ~ N(0, h_a^2 G / (2 gamma_a)) (stationary), independent of (rho, y).
 * All TOAs of all pulsars are processed in time order (ties: pulsar, then
 * TOA index).  Over dt, with x = gamma dt for each OU process:
 *   rho_n += b_p y_n + b_a a_n,  y_n *= a_p,  a_n *= a_a,
 *   a = e^-x, b = dt phi1(x);
 *   Q: (rho_n, y_n) block sigma_p,n^2 q(x_p); (rho_n, a_n) x (rho_m, a_m)
 *   blocks h_a^2 G_nm q(x_a), with q(x) = [[dt^3/3 phi4(x), dt^2/2 phi1(x)^2],
 *   [., dt phi1(2x)]] (the integrated-OU increment; the two noises are
 *   independent, so they add in rho).
 * Dense textbook algebra throughout: P = F P F^T + Q, S = P_ii + R,
 * K = P e_i / S, m += K e, P -= K S K^T.
 */
static KF_T GWB_NAME(int P, const int64_t* off, const double* t, const double* r,
                     const double* sigma, const double* equad, const double* p0,
                     const double* G, const int64_t* order, const int* psr_of, int64_t N,
                     KF_T ha2, KF_T ga, const KF_T* sig2, const KF_T* gp, const KF_T* efac,
                     int* bad)
{
    const int n = 3 * P;
    KF_T* m = calloc((size_t)n, sizeof(KF_T));
    KF_T* Pm = calloc((size_t)n * n, sizeof(KF_T));
    KF_T* F = calloc((size_t)n * n, sizeof(KF_T));
    KF_T* Q = calloc((size_t)n * n, sizeof(KF_T));
    KF_T* T = calloc((size_t)n * n, sizeof(KF_T));
    KF_T* K = calloc((size_t)n, sizeof(KF_T));
    (void)off;
    /* prior */
    for (int a = 0; a < P; ++a) {
        Pm[(3 * a) * n + 3 * a] = p0[3 * a];
        Pm[(3 * a) * n + 3 * a + 1] = p0[3 * a + 1];
        Pm[(3 * a + 1) * n + 3 * a] = p0[3 * a + 1];
        Pm[(3 * a + 1) * n + 3 * a + 1] = p0[3 * a + 2];
        for (int b = 0; b < P; ++b)
            Pm[(3 * a + 2) * n + 3 * b + 2] = ha2 * G[a * P + b] / (2.0 * ga);
    }
    double t_prev = t[order[0]];
    KF_T ll = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        const int64_t g = order[j];
        const int q = psr_of[j];
        const double dt = t[g] - t_prev;
        t_prev = t[g];
        /* transition and process noise of every pulsar over dt */
        for (int i = 0; i < n * n; ++i) { F[i] = 0.0; Q[i] = 0.0; }
        KF_T a1, a2, a4;
        KF_PHI(ga * dt, &a1, &a2, &a4);
        const KF_T aa = 1.0 - ga * dt * a1, ba = dt * a1;
        const KF_T qa00 = ha2 * (dt * dt * dt / 3.0) * a4, qa01 = ha2 * (dt * dt / 2.0) * a1 * a1,
                   qa11 = ha2 * dt * a2;
        for (int a = 0; a < P; ++a) {
            KF_T p1, p2, p4;
            KF_PHI(gp[a] * dt, &p1, &p2, &p4);
            const KF_T ap = 1.0 - gp[a] * dt * p1, bp = dt * p1;
            const int R0 = 3 * a, Y = 3 * a + 1, A = 3 * a + 2;
            F[R0 * n + R0] = 1.0; F[R0 * n + Y] = bp; F[R0 * n + A] = ba;
            F[Y * n + Y] = ap;
            F[A * n + A] = aa;
            Q[R0 * n + R0] += sig2[a] * (dt * dt * dt / 3.0) * p4;
            Q[R0 * n + Y] += sig2[a] * (dt * dt / 2.0) * p1 * p1;
            Q[Y * n + R0] += sig2[a] * (dt * dt / 2.0) * p1 * p1;
            Q[Y * n + Y] += sig2[a] * dt * p2;
            for (int b = 0; b < P; ++b) {
                const double Gab = G[a * P + b];
                const int Rb = 3 * b, Ab = 3 * b + 2;
                Q[R0 * n + Rb] += Gab * qa00;
                Q[R0 * n + Ab] += Gab * qa01;
                Q[A * n + Rb] += Gab * qa01;
                Q[A * n + Ab] += Gab * qa11;
            }
        }
        /* predict: m = F m, P = F P F^T + Q */
        for (int i = 0; i < n; ++i) {
            KF_T s = 0.0;
            for (int k = 0; k < n; ++k) s += F[i * n + k] * m[k];
            K[i] = s;
        }
        for (int i = 0; i < n; ++i) m[i] = K[i];
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < n; ++c) {
                KF_T s = 0.0;
                for (int k = 0; k < n; ++k) s += F[i * n + k] * Pm[k * n + c];
                T[i * n + c] = s;
            }
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < n; ++c) {
                KF_T s = Q[i * n + c];
                for (int k = 0; k < n; ++k) s += T[i * n + k] * F[c * n + k];
                Pm[i * n + c] = s;
            }
        /* innovate */
        const int i0 = 3 * q;
        const KF_T Rk = efac[q] * efac[q] * (sigma[g] * sigma[g]) + equad[q] * equad[q];
        const KF_T e = r[g] - m[i0];
        const KF_T S = Pm[i0 * n + i0] + Rk;
        if (!(KF_RE(S) > 0.0)) *bad = 1;
        /* update */
        for (int i = 0; i < n; ++i) K[i] = Pm[i * n + i0] / S;
        for (int i = 0; i < n; ++i) m[i] += K[i] * e;
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < n; ++c) T[i * n + c] = Pm[i * n + c] - K[i] * S * K[c];
        for (int i = 0; i < n * n; ++i) Pm[i] = T[i];
        ll += -0.5 * (KF_LOG2PI + KF_LOG(S) + e * e / S);
    }
    free(m); free(Pm); free(F); free(Q); free(T); free(K);
    return ll;
}
