/*
 * phi-functions of the Ornstein-Uhlenbeck transition, for KF_T = double or
 * double complex (included by each instantiation of the filter bodies).
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle.
 *
 * With x = gamma dt: phi1(x) = (1 - e^-x)/x, phi1(2x), and
 * phi4(x) = 3 (x - 2 (1 - e^-x) + (1 - e^-2x)/2) / x^3, all -> 1 as x -> 0;
 * Taylor series below x = 0.5, closed forms above.
 */
static void KF_PHI(KF_T x, KF_T* p1, KF_T* p2, KF_T* p4)
{
    if (KF_RE(x) < 0.5) {
        /* Taylor series, 22 terms: phi1 = sum (-x)^m/(m+1)!,
           phi4 = sum 3 (-1)^(m+3) (2 - 2^(m+2)) / (m+3)! x^m */
        KF_T s1 = 0.0, s2 = 0.0, s4 = 0.0;
        for (int m = 21; m >= 0; --m) {
            double f1 = 1.0, f4 = 1.0;
            for (int i = 2; i <= m + 1; ++i) f1 *= i;
            for (int i = 2; i <= m + 3; ++i) f4 *= i;
            double c1 = ((m & 1) ? -1.0 : 1.0) / f1;
            double c4 = 3.0 * (((m + 3) & 1) ? -1.0 : 1.0) * (2.0 - pow(2.0, m + 2)) / f4;
            s1 = s1 * x + c1;
            s2 = s2 * (2.0 * x) + c1;
            s4 = s4 * x + c4;
        }
        *p1 = s1; *p2 = s2; *p4 = s4;
    } else {
        KF_T e1 = KF_EXP(-x), e2 = KF_EXP(-2.0 * x);
        *p1 = (1.0 - e1) / x;
        *p2 = (1.0 - e2) / (2.0 * x);
        *p4 = 3.0 * (x - 2.0 * (1.0 - e1) + 0.5 * (1.0 - e2)) / (x * x * x);
    }
}

