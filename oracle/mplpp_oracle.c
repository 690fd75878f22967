/*
 * mplpp_oracle.c -- plain, slow FP64 reference of MPLP++ (Tourani et al.,
 * "MPLP++: Fast, Parallel Dual Block-Coordinate Ascent for Dense Graphical
 * Models").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this file.  The product path
 * (the CUDA library) never calls it and shares no code with it.
 *
 * Representation ("table form"): the oracle keeps the CURRENT reparametrized
 * cost vector theta^phi itself, i.e. one unary vector per node and one full
 * L_u x L_v pairwise table per edge, and overwrites them in place, exactly as
 * Sec. 4 (Def. 1 and the equation after it) describes a BCA update:
 *     theta_u := theta^gamma_u, theta_v := theta^gamma_v,
 *     theta_uv := g_uv - theta^gamma_u - theta^gamma_v.
 * No messages, no aggregates, no blocking, no fusion.
 *
 * Indexing: nodes 0..n-1 with label counts L[u]; unaries concatenated node by
 * node (uoff[u] = sum_{w<u} L[w]); edges e = (eu[e], ev[e]) with eu < ev
 * (Sec. 3 Notation: uv in E means u < v); the table of edge e is row-major
 * with rows indexed by the labels of eu[e] and columns by those of ev[e],
 * stored at poff[e] = sum_{f<e} L[eu[f]] * L[ev[f]].
 *
 * Ties in argmin are broken towards the lowest index everywhere.
 *
 * Parity pins (tests/test_oracle_*.py): worked example of Prop. 3 (appendix,
 * proof that H is not monotonous), update invariants of Def. 1 / eq. (H),
 * dominance H >= M >= U (Prop. 2), one-iteration dominance (Thm. 2),
 * monotone dual (Lemma B.4), energy invariance under reparametrization
 * (Sec. 3 Dual Problem), D <= brute-force MAP, single-edge exactness
 * (Prop. 1), convergence to the MAP energy on trees, and central finite
 * differences for the gradient.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define ORC_RULE_U 0 /* eq. (U): uniform update                       */
#define ORC_RULE_M 1 /* eq. (M): MPLP update                          */
#define ORC_RULE_H 2 /* eq. (H): MPLP++ / handshake update            */

/* ---------------------------------------------------------------------- */
/* One BCA update of edge uv (Sec. 4, Def. 2 and eqs. (U), (M), (H)).     */
/*   th_u [Lu], th_v [Lv], th_uv [Lu*Lv]: current reparametrized costs,   */
/*   overwritten with the result.                                         */
/*   t1, s2, t3 (rule H only, may be NULL): argmins of the three          */
/*   minimizations, used by the reverse-mode gradient.                    */
/* Returns 0, or -1 on allocation failure.                                */
/* ---------------------------------------------------------------------- */
int orc_update_edge(int rule, int Lu, int Lv, double *th_u, double *th_v,
                    double *th_uv, int *t1, int *s2, int *t3)
{
    double *g = (double *)malloc(sizeof(double) * (size_t)Lu * (size_t)Lv);
    double *nu = (double *)malloc(sizeof(double) * (size_t)Lu);
    double *nv = (double *)malloc(sizeof(double) * (size_t)Lv);
    if (!g || !nu || !nv) {
        free(g); free(nu); free(nv);
        return -1;
    }
    /* aggregated cost g_uv(s,t) = theta_uv(s,t) + theta_u(s) + theta_v(t)  (Sec. 4) */
    for (int s = 0; s < Lu; ++s)
        for (int t = 0; t < Lv; ++t)
            g[(size_t)s * Lv + t] = th_uv[(size_t)s * Lv + t] + th_u[s] + th_v[t];

    if (rule == ORC_RULE_U) {
        /* eq. (U): both unaries := 1/2 min_{s',t'} g(s',t') */
        double m = INFINITY;
        for (size_t i = 0; i < (size_t)Lu * Lv; ++i)
            if (g[i] < m) m = g[i];
        for (int s = 0; s < Lu; ++s) nu[s] = 0.5 * m;
        for (int t = 0; t < Lv; ++t) nv[t] = 0.5 * m;
    } else if (rule == ORC_RULE_M) {
        /* eq. (M): theta_u(s) := 1/2 min_t g(s,t);  theta_v(t) := 1/2 min_s g(s,t) */
        for (int s = 0; s < Lu; ++s) {
            double m = INFINITY;
            for (int t = 0; t < Lv; ++t)
                if (g[(size_t)s * Lv + t] < m) m = g[(size_t)s * Lv + t];
            nu[s] = 0.5 * m;
        }
        for (int t = 0; t < Lv; ++t) {
            double m = INFINITY;
            for (int s = 0; s < Lu; ++s)
                if (g[(size_t)s * Lv + t] < m) m = g[(size_t)s * Lv + t];
            nv[t] = 0.5 * m;
        }
    } else {
        /* eq. (H) in its three-minimization form (Sec. 4, text after eq. (H)):
         *   a(s) = 1/2 min_t g(s,t)           (the MPLP value of theta_u)
         *   b(t) = min_s [g(s,t) - a(s)]      (new theta_v)
         *   c(s) = min_t [g(s,t) - b(t)]      (new theta_u)                 */
        double *a = (double *)malloc(sizeof(double) * (size_t)Lu);
        if (!a) {
            free(g); free(nu); free(nv);
            return -1;
        }
        for (int s = 0; s < Lu; ++s) {
            double m = INFINITY;
            int am = 0;
            for (int t = 0; t < Lv; ++t)
                if (g[(size_t)s * Lv + t] < m) { m = g[(size_t)s * Lv + t]; am = t; }
            a[s] = 0.5 * m;
            if (t1) t1[s] = am;
        }
        for (int t = 0; t < Lv; ++t) {
            double m = INFINITY;
            int am = 0;
            for (int s = 0; s < Lu; ++s) {
                double x = g[(size_t)s * Lv + t] - a[s];
                if (x < m) { m = x; am = s; }
            }
            nv[t] = m;
            if (s2) s2[t] = am;
        }
        for (int s = 0; s < Lu; ++s) {
            double m = INFINITY;
            int am = 0;
            for (int t = 0; t < Lv; ++t) {
                double x = g[(size_t)s * Lv + t] - nv[t];
                if (x < m) { m = x; am = t; }
            }
            nu[s] = m;
            if (t3) t3[s] = am;
        }
        free(a);
    }
    /* reparametrized result (Sec. 4): theta^gamma_uv = g - theta^gamma_u - theta^gamma_v */
    for (int s = 0; s < Lu; ++s) th_u[s] = nu[s];
    for (int t = 0; t < Lv; ++t) th_v[t] = nv[t];
    for (int s = 0; s < Lu; ++s)
        for (int t = 0; t < Lv; ++t)
            th_uv[(size_t)s * Lv + t] = g[(size_t)s * Lv + t] - nu[s] - nv[t];
    free(g); free(nu); free(nv);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Dual lower bound D(theta^phi) (Sec. 3, eq. LP-lower-bound):            */
/*   sum_u min_s theta_u(s) + sum_uv min_{s,t} theta_uv(s,t).             */
/* ---------------------------------------------------------------------- */
double orc_bound(int n, const int *L, const long *uoff, int E, const int *eu,
                 const int *ev, const long *poff, const double *th_u,
                 const double *th_uv)
{
    double D = 0.0;
    for (int u = 0; u < n; ++u) {
        double m = INFINITY;
        for (int s = 0; s < L[u]; ++s)
            if (th_u[uoff[u] + s] < m) m = th_u[uoff[u] + s];
        D += m;
    }
    for (int e = 0; e < E; ++e) {
        long sz = (long)L[eu[e]] * L[ev[e]];
        double m = INFINITY;
        for (long i = 0; i < sz; ++i)
            if (th_uv[poff[e] + i] < m) m = th_uv[poff[e] + i];
        D += m;
    }
    return D;
}

/* ---------------------------------------------------------------------- */
/* T BCA iterations (Sec. 5: an iteration applies the update to all edges */
/* in a chosen order; Sec. 6: the order is the concatenation of the       */
/* matchings of the edge schedule).  order[0..n_order) lists edge ids in  */
/* visiting order; one iteration visits them all once.                    */
/* D_hist (may be NULL) receives D after each iteration.                  */
/* ---------------------------------------------------------------------- */
int orc_run(int rule, int n, const int *L, const long *uoff, int E,
            const int *eu, const int *ev, const long *poff, int n_order,
            const int *order, int T, double *th_u, double *th_uv,
            double *D_hist)
{
    for (int it = 0; it < T; ++it) {
        for (int k = 0; k < n_order; ++k) {
            int e = order[k];
            int u = eu[e], v = ev[e];
            if (orc_update_edge(rule, L[u], L[v], th_u + uoff[u], th_u + uoff[v],
                                th_uv + poff[e], NULL, NULL, NULL))
                return -1;
        }
        if (D_hist)
            D_hist[it] = orc_bound(n, L, uoff, E, eu, ev, poff, th_u, th_uv);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* The same T iterations with the edges of one matching updated by       */
/* several host threads (Sec. 6: the edges of a matching share no node,   */
/* so their updates touch disjoint data and commute).  Matching k is      */
/* order[moff[k] .. moff[k+1]); matchings run in order.  Every update is  */
/* the same sequence of FP64 operations on the same data as in orc_run,   */
/* so the result equals orc_run's bit for bit for any thread count.       */
/* threads <= 0: the OpenMP default.  Returns -1 on allocation failure,   */
/* -2 if an edge of a matching shares a node with another one.            */
/* ---------------------------------------------------------------------- */
int orc_run_parallel(int rule, int n, const int *L, const long *uoff, int E,
                     const int *eu, const int *ev, const long *poff,
                     int n_match, const int *moff, const int *order, int T,
                     double *th_u, double *th_uv, int threads)
{
    int *seen = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!seen) return -1;
    for (int u = 0; u < n; ++u) seen[u] = -1;
    for (int k = 0; k < n_match; ++k)
        for (int i = moff[k]; i < moff[k + 1]; ++i) {
            int e = order[i];
            if (seen[eu[e]] == k || seen[ev[e]] == k) {
                free(seen);
                return -2;
            }
            seen[eu[e]] = k;
            seen[ev[e]] = k;
        }
    free(seen);
    (void)E;
    int failed = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    for (int it = 0; it < T && !failed; ++it)
        for (int k = 0; k < n_match && !failed; ++k) {
            int lo = moff[k], hi = moff[k + 1];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(|| : failed)
#endif
            for (int i = lo; i < hi; ++i) {
                int e = order[i];
                int u = eu[e], v = ev[e];
                if (orc_update_edge(rule, L[u], L[v], th_u + uoff[u], th_u + uoff[v],
                                    th_uv + poff[e], NULL, NULL, NULL))
                    failed = 1;
            }
        }
    return failed ? -1 : 0;
}

/* Threads the OpenMP runtime uses by default (1 without OpenMP). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Energy E(y|theta) (Sec. 3, eq. energy-min).                            */
/* ---------------------------------------------------------------------- */
double orc_energy(int n, const int *L, const long *uoff, int E, const int *eu,
                  const int *ev, const long *poff, const double *th_u,
                  const double *th_uv, const int *y)
{
    double En = 0.0;
    for (int u = 0; u < n; ++u) En += th_u[uoff[u] + y[u]];
    for (int e = 0; e < E; ++e)
        En += th_uv[poff[e] + (long)y[eu[e]] * L[ev[e]] + y[ev[e]]];
    return En;
}

/* Edges grouped by their larger endpoint ev, each group sorted by the    */
/* smaller endpoint eu: in-edges of u are eid[cnt[u] .. cnt[u+1]).        */
static int orc_in_edges(int n, int E, const int *eu, const int *ev, int **eid_out,
                        int **cnt_out)
{
    int *eid = (int *)malloc(sizeof(int) * (size_t)(E > 0 ? E : 1));
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
    int *fill = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!eid || !cnt || !fill) {
        free(eid); free(cnt); free(fill);
        return -1;
    }
    for (int e = 0; e < E; ++e) cnt[ev[e] + 1]++;
    for (int u = 0; u < n; ++u) cnt[u + 1] += cnt[u];
    for (int u = 0; u < n; ++u) fill[u] = cnt[u];
    for (int e = 0; e < E; ++e) eid[fill[ev[e]]++] = e;
    free(fill);
    for (int u = 0; u < n; ++u) /* insertion sort by eu */
        for (int i = cnt[u] + 1; i < cnt[u + 1]; ++i)
            for (int j = i; j > cnt[u] && eu[eid[j - 1]] > eu[eid[j]]; --j) {
                int tmp = eid[j]; eid[j] = eid[j - 1]; eid[j - 1] = tmp;
            }
    *eid_out = eid;
    *cnt_out = cnt;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Primal rounding (Sec. 4, Primal Rounding): nodes in increasing order,  */
/*   x_u in argmin_s [theta_u(s) + sum_{v<u, vu in E} theta_vu(x_v, s)]   */
/* on the reparametrized costs.  The sum runs over the earlier            */
/* neighbours v in increasing order of v.  margin[u] (may be NULL)        */
/* receives (second smallest - smallest) of the minimized objective, or   */
/* +inf when L_u == 1.                                                    */
/* ---------------------------------------------------------------------- */
int orc_round(int n, const int *L, const long *uoff, int E, const int *eu,
              const int *ev, const long *poff, const double *th_u,
              const double *th_uv, int *x, double *margin)
{
    int Lmax = 1;
    for (int u = 0; u < n; ++u) if (L[u] > Lmax) Lmax = L[u];
    double *obj = (double *)malloc(sizeof(double) * (size_t)Lmax);
    int *eid = NULL, *cnt = NULL;
    if (!obj || orc_in_edges(n, E, eu, ev, &eid, &cnt)) {
        free(obj);
        return -1;
    }
    for (int u = 0; u < n; ++u) {
        for (int s = 0; s < L[u]; ++s) obj[s] = th_u[uoff[u] + s];
        for (int i = cnt[u]; i < cnt[u + 1]; ++i) {
            int e = eid[i];
            int v = eu[e];
            for (int s = 0; s < L[u]; ++s)
                obj[s] += th_uv[poff[e] + (long)x[v] * L[u] + s];
        }
        int best = 0;
        for (int s = 1; s < L[u]; ++s) if (obj[s] < obj[best]) best = s;
        x[u] = best;
        if (margin) {
            double second = INFINITY;
            for (int s = 0; s < L[u]; ++s)
                if (s != best && obj[s] < second) second = obj[s];
            margin[u] = second - obj[best];
        }
    }
    free(obj); free(eid); free(cnt);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Gradient of D after T iterations of rule H with respect to the         */
/* ORIGINAL costs (theta_u, theta_uv), by reverse-mode differentiation of */
/* the table-form iteration.  D is piecewise linear; inside a linear      */
/* piece its gradient follows the recorded argmins (lowest-index ties).   */
/*                                                                        */
/* Forward (per update, as in orc_update_edge, rule H):                   */
/*   g = th_uv + th_u (+) th_v                                            */
/*   a(s) = 1/2 g(s, t1(s));  b(t) = g(s2(t), t) - a(s2(t));              */
/*   c(s) = g(s, t3(s)) - b(t3(s));                                       */
/*   th_u' = c, th_v' = b, th_uv' = g - c (+) b.                          */
/* Reverse: given adjoints U', V', W' of th_u', th_v', th_uv':            */
/*   cbar(s) = U'(s) - sum_t W'(s,t);  bbar(t) = V'(t) - sum_s W'(s,t);   */
/*   gbar = W';  gbar(s,t3(s)) += cbar(s),  bbar(t3(s)) -= cbar(s);       */
/*   abar = 0;   gbar(s2(t),t) += bbar(t),  abar(s2(t)) -= bbar(t);       */
/*   gbar(s,t1(s)) += abar(s)/2;                                          */
/*   adjoint of th_uv := gbar, of th_u := row sums, of th_v := col sums.  */
/* The initial adjoint is that of D itself: 1 at the (lowest-index)       */
/* argmin of every unary vector and every pairwise table.                 */
/* Outputs: grad_u [sum L], grad_uv [sum Lu*Lv], *D_out = final D.        */
/* ---------------------------------------------------------------------- */
int orc_grad(int n, const int *L, const long *uoff, int E, const int *eu,
             const int *ev, const long *poff, int n_order, const int *order,
             int T, const double *th0_u, const double *th0_uv, double *grad_u,
             double *grad_uv, double *D_out)
{
    long NU = uoff[n];
    long NP = poff[E];
    /* argmin records: per visit, 2*Lu + Lv ints */
    long per_iter = 0;
    for (int k = 0; k < n_order; ++k) {
        int e = order[k];
        per_iter += 2L * L[eu[e]] + L[ev[e]];
    }
    double *th_u = (double *)malloc(sizeof(double) * (size_t)(NU > 0 ? NU : 1));
    double *th_uv = (double *)malloc(sizeof(double) * (size_t)(NP > 0 ? NP : 1));
    int *rec = (int *)malloc(sizeof(int) * (size_t)(per_iter * T > 0 ? per_iter * T : 1));
    int Lmax = 1;
    for (int u = 0; u < n; ++u) if (L[u] > Lmax) Lmax = L[u];
    double *gbar = (double *)malloc(sizeof(double) * (size_t)Lmax * Lmax);
    double *cbar = (double *)malloc(sizeof(double) * (size_t)Lmax);
    double *bbar = (double *)malloc(sizeof(double) * (size_t)Lmax);
    double *abar = (double *)malloc(sizeof(double) * (size_t)Lmax);
    if (!th_u || !th_uv || !rec || !gbar || !cbar || !bbar || !abar) {
        free(th_u); free(th_uv); free(rec); free(gbar); free(cbar); free(bbar); free(abar);
        return -1;
    }
    memcpy(th_u, th0_u, sizeof(double) * (size_t)NU);
    memcpy(th_uv, th0_uv, sizeof(double) * (size_t)NP);

    /* forward, recording argmins */
    long pos = 0;
    for (int it = 0; it < T; ++it)
        for (int k = 0; k < n_order; ++k) {
            int e = order[k];
            int u = eu[e], v = ev[e];
            int Lu = L[u], Lv = L[v];
            int *t1 = rec + pos, *s2 = rec + pos + Lu, *t3 = rec + pos + Lu + Lv;
            if (orc_update_edge(ORC_RULE_H, Lu, Lv, th_u + uoff[u], th_u + uoff[v],
                                th_uv + poff[e], t1, s2, t3)) {
                free(th_u); free(th_uv); free(rec); free(gbar); free(cbar); free(bbar); free(abar);
                return -1;
            }
            pos += 2L * Lu + Lv;
        }
    if (D_out) *D_out = orc_bound(n, L, uoff, E, eu, ev, poff, th_u, th_uv);

    /* adjoint of D at the final state */
    memset(grad_u, 0, sizeof(double) * (size_t)NU);
    memset(grad_uv, 0, sizeof(double) * (size_t)NP);
    for (int u = 0; u < n; ++u) {
        int best = 0;
        for (int s = 1; s < L[u]; ++s)
            if (th_u[uoff[u] + s] < th_u[uoff[u] + best]) best = s;
        grad_u[uoff[u] + best] += 1.0;
    }
    for (int e = 0; e < E; ++e) {
        long sz = (long)L[eu[e]] * L[ev[e]];
        long best = 0;
        for (long i = 1; i < sz; ++i)
            if (th_uv[poff[e] + i] < th_uv[poff[e] + best]) best = i;
        grad_uv[poff[e] + best] += 1.0;
    }

    /* reverse sweep over all visits */
    for (int it = T - 1; it >= 0; --it)
        for (int k = n_order - 1; k >= 0; --k) {
            int e = order[k];
            int u = eu[e], v = ev[e];
            int Lu = L[u], Lv = L[v];
            pos -= 2L * Lu + Lv;
            const int *t1 = rec + pos, *s2 = rec + pos + Lu, *t3 = rec + pos + Lu + Lv;
            double *W = grad_uv + poff[e];
            double *Ub = grad_u + uoff[u];
            double *Vb = grad_u + uoff[v];
            for (int s = 0; s < Lu; ++s) {
                double rs = 0.0;
                for (int t = 0; t < Lv; ++t) rs += W[(size_t)s * Lv + t];
                cbar[s] = Ub[s] - rs;
            }
            for (int t = 0; t < Lv; ++t) {
                double cs = 0.0;
                for (int s = 0; s < Lu; ++s) cs += W[(size_t)s * Lv + t];
                bbar[t] = Vb[t] - cs;
            }
            for (size_t i = 0; i < (size_t)Lu * Lv; ++i) gbar[i] = W[i];
            for (int s = 0; s < Lu; ++s) {
                gbar[(size_t)s * Lv + t3[s]] += cbar[s];
                bbar[t3[s]] -= cbar[s];
            }
            for (int s = 0; s < Lu; ++s) abar[s] = 0.0;
            for (int t = 0; t < Lv; ++t) {
                gbar[(size_t)s2[t] * Lv + t] += bbar[t];
                abar[s2[t]] -= bbar[t];
            }
            for (int s = 0; s < Lu; ++s) gbar[(size_t)s * Lv + t1[s]] += 0.5 * abar[s];
            for (size_t i = 0; i < (size_t)Lu * Lv; ++i) W[i] = gbar[i];
            for (int s = 0; s < Lu; ++s) {
                double rs = 0.0;
                for (int t = 0; t < Lv; ++t) rs += gbar[(size_t)s * Lv + t];
                Ub[s] = rs;
            }
            for (int t = 0; t < Lv; ++t) {
                double cs = 0.0;
                for (int s = 0; s < Lu; ++s) cs += gbar[(size_t)s * Lv + t];
                Vb[t] = cs;
            }
        }
    free(th_u); free(th_uv); free(rec); free(gbar); free(cbar); free(bbar); free(abar);
    return 0;
}
