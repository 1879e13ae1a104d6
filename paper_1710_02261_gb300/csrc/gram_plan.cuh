// gram_plan.cuh -- which Gram outputs a thread of a run updates, and from
// which Delta elements (Eqs. rowB, rowC).  Plain constexpr C++ (no device
// code), so host tests can check the plan.
//
// The outputs of one entry are the upper triangle of delta delta^T, row-major
// over j <= k (output g = (j, k)), then x * delta_k (output NTRI + k).
#pragma once

namespace ptk {

// upper-triangle output index q -> (j, k), row-major over j <= k
template <int J>
struct Tri {
    int j[J * (J + 1) / 2], k[J * (J + 1) / 2];
    constexpr Tri() : j(), k() {
        int q = 0;
        for (int a = 0; a < J; ++a)
            for (int b = a; b < J; ++b) {
                j[q] = a;
                k[q] = b;
                ++q;
            }
    }
};

// Which outputs a thread updates together, and from which Delta elements.
// Output g is the product d[pa] * d[pb] (B_jk: d[j] * d[k]; c_k: d[k] * x with
// x = d[J]).  Pairs are chosen so that their operands are neighbouring
// elements where possible: B_{j,k} with B_{j+1,k+1} (j, k even) takes
// (d[j], d[j+1]) times (d[k], d[k+1]); c_k with c_{k+1} takes (d[k], d[k+1])
// times (x, x); the rest are paired in output order.  Pairs are dealt to the
// four threads of a run in turn.
template <int J>
struct PackPlan {
    static constexpr int NTRI = J * (J + 1) / 2, NOUT = NTRI + J;
    static constexpr int MAXP = (NOUT + 1) / 2;
    static constexpr int PMAX = (MAXP + 3) / 4;
    int np[4];
    int g0[4][PMAX], g1[4][PMAX], a0[4][PMAX], a1[4][PMAX], b0[4][PMAX], b1[4][PMAX];
    static constexpr int gtri(int j, int k) { return j * J - j * (j - 1) / 2 + (k - j); }
    static constexpr int opa(int g) {
        if (g >= NTRI) return g - NTRI;
        int j = 0, first = 0;
        while (g >= first + (J - j)) {
            first += J - j;
            ++j;
        }
        return j;
    }
    static constexpr int opb(int g) {
        if (g >= NTRI) return J;
        int j = 0, first = 0;
        while (g >= first + (J - j)) {
            first += J - j;
            ++j;
        }
        return j + (g - first);
    }
    constexpr PackPlan() : np(), g0(), g1(), a0(), a1(), b0(), b1() {
        int P0[MAXP] = {}, P1[MAXP] = {};
        bool used[NOUT] = {};
        int n = 0;
        for (int j = 0; j + 1 < J; j += 2)
            for (int k = j; k + 1 < J; k += 2) {
                P0[n] = gtri(j, k);
                P1[n] = gtri(j + 1, k + 1);
                used[P0[n]] = used[P1[n]] = true;
                ++n;
            }
        for (int k = 0; k + 1 < J; k += 2) {
            P0[n] = NTRI + k;
            P1[n] = NTRI + k + 1;
            used[P0[n]] = used[P1[n]] = true;
            ++n;
        }
        int pend = -1;
        for (int g = 0; g < NOUT; ++g) {
            if (used[g]) continue;
            if (pend < 0) {
                pend = g;
                continue;
            }
            P0[n] = pend;
            P1[n] = g;
            ++n;
            pend = -1;
        }
        if (pend >= 0) {
            P0[n] = pend;
            P1[n] = -1;
            ++n;
        }
        for (int i = 0; i < n; ++i) {
            const int p = i % 4, q = np[p]++;
            g0[p][q] = P0[i];
            g1[p][q] = P1[i];
            a0[p][q] = opa(P0[i]);
            b0[p][q] = opb(P0[i]);
            a1[p][q] = P1[i] >= 0 ? opa(P1[i]) : a0[p][q];
            b1[p][q] = P1[i] >= 0 ? opb(P1[i]) : b0[p][q];
        }
    }
};

}  // namespace ptk
