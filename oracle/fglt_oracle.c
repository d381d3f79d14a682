/*
 * Plain CPU oracle of the Fast Graphlet Transform (Floros, Pitsianis, Sun,
 * "Fast Graphlet Transform of Sparse Graphs").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this code;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code with the CUDA path.
 *
 * Input: a simple undirected graph as a symmetric CSR (int64 row pointers,
 * int32 column indices, sorted neighbour lists, 0-based vertex ids).
 * Output: per vertex the 16 raw frequencies f^(v) of Table I and the 16 net
 * frequencies f(v) = U16^{-1} f^(v) of Table II, all in int64.
 *
 * The computation follows the paper's steps literally and in order:
 *   1. p1 = d1 = A e and p2 = A p1 - c2 with c2 = d1            (eq. p2, Sec. 3.1)
 *   2. C3 = A o A^2 per directed edge, c3 = C3 e / 2             (Lemma 2, Sec. 3.1)
 *   3. p3 = A p2 - p1 o (p1 - 1) - 2 c3                          (Lemma on p3, Sec. 4.1)
 *   4. the elementwise and SpMV rows of Table I                  (Sec. 4.1, 4.2, Table I)
 *   5. P2 row of each vertex; c4 = C4,2 e / 2 with C4,2 = P2 o (P2 - 1),
 *      and D4,3 = A o C4,2                                       (Lemma on c4, Sec. 4.1; Sec. 4.3)
 *   6. D4,c = A o (A (C3 - A)), d^13 = D4,c e / 2                (Sec. 4.3)
 *   7. T = A o [q_ij^T A q_ij], q_ij = a_i o a_j, d^15 = T e / 6 (Sec. 4.3)
 *   8. net = U16^{-1} raw by back substitution on U16 as printed (Table II)
 * Set intersections are plain sorted merges (or binary searches where one side
 * is much shorter); no other blocking, fusion or reordering is done.
 *
 * Readings of the paper taken here:
 *  - every "-" in Table I is the rectified difference max(x - y, 0) (Sec. 1,
 *    notation); for the quantities below it never clips a count, so the code
 *    clips only where a factor can be negative (p1 - 2 at degree 1 or 0) and
 *    the product would otherwise be non-zero; see rsub().
 *  - the in-text tri-node net formulas of Sec. 3.2 have swapped coefficients;
 *    net values come only from Table II (back substitution).
 *  - T(i,j) = q_ij^T A q_ij, i.e. twice the number of 4-cliques on edge ij,
 *    and d^15 = T e / 6 (Sec. 4.3 definition; the proof sketch's constants are
 *    not used).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
#include <time.h>
#endif

typedef int64_t i64;
typedef int32_t i32;

#define NG 16

/* Wall clock in seconds (measurement only: the CPU-baseline leg of the
 * benchmark reads per-row times to extrapolate from a vertex sample). */
static double wall_s(void) {
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return (double)clock() / CLOCKS_PER_SEC;
#endif
}

/* Rectified difference of the paper's notation paragraph: max(x - y, 0). */
static inline i64 rsub(i64 x, i64 y) { return x > y ? x - y : 0; }

/* Table II: U16, row k = raw frequency d^_k, column l = net frequency d_l. */
static const i64 U16[NG][NG] = {
    /*        0  1  2  3  4  5  6  7  8  9 10 11 12 13 14 15 */
    /* 0 */ { 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0 },
    /* 1 */ { 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0 },
    /* 2 */ { 0, 0, 1, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0 },
    /* 3 */ { 0, 0, 0, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0 },
    /* 4 */ { 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0 },
    /* 5 */ { 0, 0, 0, 0, 0, 1, 0, 0, 0, 2, 1, 0, 2, 4, 2, 6 },
    /* 6 */ { 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 1, 2, 2, 2, 4, 6 },
    /* 7 */ { 0, 0, 0, 0, 0, 0, 0, 1, 0, 1, 1, 0, 0, 2, 1, 3 },
    /* 8 */ { 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 1, 1 },
    /* 9 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 2, 0, 3 },
    /*10 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 2, 2, 6 },
    /*11 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 2, 3 },
    /*12 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 3 },
    /*13 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 3 },
    /*14 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 3 },
    /*15 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1 },
};

/* Exposes Table II to the tests (they check it against Fig. 2 independently). */
void oracle_u16(i64* out /* 16*16 row-major */) { memcpy(out, U16, sizeof U16); }

typedef struct {
    i64 n;
    const i64* rp;
    const i32* ci;
} graph;

static inline i64 deg(const graph* g, i64 i) { return g->rp[i + 1] - g->rp[i]; }

/* Position of key in the sorted list a[0..na), or -1. */
static i64 find_pos(const i32* a, i64 na, i32 key) {
    i64 lo = 0, hi = na;
    while (lo < hi) {
        i64 mid = lo + (hi - lo) / 2;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < na && a[lo] == key) ? lo : -1;
}

/* |N(i) ∩ N(j)| of two sorted lists: a sorted merge, or, when one list is
 * much longer, a binary search of each element of the shorter one. */
static i64 merge_count(const i32* a, i64 na, const i32* b, i64 nb) {
    if (na > 8 * nb || nb > 8 * na) {
        const i32* s = na < nb ? a : b;
        const i32* l = na < nb ? b : a;
        i64 ns = na < nb ? na : nb, nl = na < nb ? nb : na, c = 0;
        for (i64 x = 0; x < ns; x++) c += find_pos(l, nl, s[x]) >= 0;
        return c;
    }
    i64 x = 0, y = 0, c = 0;
    while (x < na && y < nb) {
        if (a[x] < b[y]) x++;
        else if (a[x] > b[y]) y++;
        else { c++; x++; y++; }
    }
    return c;
}

/* The common elements of two sorted lists a[0..na), b[0..nb): writes each
 * common value to val[] and its position in b to posb[], in increasing order,
 * and returns how many there are. A sorted merge, or, when one list is much
 * longer, a binary search of each element of the shorter one. */
static i64 intersect(const i32* a, i64 na, const i32* b, i64 nb, i64* val, i64* posb) {
    i64 c = 0;
    if (na > 8 * nb) {
        for (i64 y = 0; y < nb; y++)
            if (find_pos(a, na, b[y]) >= 0) { val[c] = b[y]; posb[c] = y; c++; }
    } else if (nb > 8 * na) {
        for (i64 x = 0; x < na; x++) {
            i64 y = find_pos(b, nb, a[x]);
            if (y >= 0) { val[c] = a[x]; posb[c] = y; c++; }
        }
    } else {
        i64 x = 0, y = 0;
        while (x < na && y < nb) {
            if (a[x] < b[y]) x++;
            else if (a[x] > b[y]) y++;
            else { val[c] = a[x]; posb[c] = y; c++; x++; y++; }
        }
    }
    return c;
}

/* A(k, l) for a vertex pair. */
static int adjacent(const graph* g, i64 k, i32 l) {
    return find_pos(g->ci + g->rp[k], deg(g, k), l) >= 0;
}

/* ---------------------------------------------------------------------------
 * Step 2: C3(i,j) = (A o A^2)(i,j) = a_i^T a_j for every directed edge, stored
 * aligned with the column indices.
 * ------------------------------------------------------------------------- */
static void step_C3(const graph* g, i64* C3, const unsigned char* rows_needed, int nthreads, double* t_c3) {
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (i64 i = 0; i < g->n; i++) {
        if (rows_needed && !rows_needed[i]) continue;
        const double t0 = t_c3 ? wall_s() : 0.0;
        const i32* Ni = g->ci + g->rp[i];
        i64 di = deg(g, i);
        for (i64 e = g->rp[i]; e < g->rp[i + 1]; e++) {
            i64 j = g->ci[e];
            C3[e] = merge_count(Ni, di, g->ci + g->rp[j], deg(g, j));
        }
        if (t_c3) t_c3[i] = wall_s() - t0;
    }
}

/* ---------------------------------------------------------------------------
 * Steps 5-7 for one vertex i. acc is a zeroed int64 scratch of length n and
 * touched a scratch of length 2n; both are left zeroed / unused on return.
 * ------------------------------------------------------------------------- */
typedef struct { i64 c4, d43, d4c, T; } quad_terms;

static quad_terms quad_row(const graph* g, i64 i, const i64* C3, i64* acc, i64* touched) {
    quad_terms r = {0, 0, 0, 0};
    const i32* Ni = g->ci + g->rp[i];
    i64 di = deg(g, i);

    /* Step 5: row i of P2 = A^2 - diag(d1): P2(i,l) = #{k : A(i,k) A(k,l)} for l != i. */
    i64 nt = 0;
    for (i64 x = 0; x < di; x++) {
        i64 k = Ni[x];
        for (i64 e = g->rp[k]; e < g->rp[k + 1]; e++) {
            i64 l = g->ci[e];
            if (l == i) continue;
            if (acc[l] == 0) touched[nt++] = l;
            acc[l]++;
        }
    }
    /* C4,2(i,l) = P2(i,l) (P2(i,l) - 1); c4(i) = sum_l C4,2(i,l) / 2. */
    i64 c42 = 0;
    for (i64 t = 0; t < nt; t++) {
        i64 p = acc[touched[t]];
        c42 += p * (p - 1);
    }
    r.c4 = c42 / 2;
    /* D4,3 = A o C4,2: only the entries on the edges of i. */
    i64 d43 = 0;
    for (i64 x = 0; x < di; x++) {
        i64 p = acc[Ni[x]];
        d43 += p * (p - 1);
    }
    r.d43 = d43; /* row sum of D4,3; halved by the caller (Table I) */
    for (i64 t = 0; t < nt; t++) acc[touched[t]] = 0;

    /* Step 6: D4,c(i,j) = sum_{k in N(i)} (C3(k,j) - A(k,j))_+ for j in N(i).
     * C3(k,j) is non-zero only on edges, so the terms are C3(k,j) - 1 over the
     * common neighbours k of i and j; the intersection of N(i) and N(j) yields
     * k together with its position in N(j), where C3(j,k) = C3(k,j) is stored. */
    i64* q = touched;       /* common neighbours (reuses the scratch) */
    i64* qpos = touched + g->n; /* their positions in N(j) */
    i64 d4c = 0;
    for (i64 x = 0; x < di; x++) {
        i64 j = Ni[x];
        i64 nq = intersect(Ni, di, g->ci + g->rp[j], deg(g, j), q, qpos);
        for (i64 s = 0; s < nq; s++) d4c += rsub(C3[g->rp[j] + qpos[s]], 1);
    }
    r.d4c = d4c; /* row sum of D4,c; halved by the caller */

    /* Step 7: T(i,j) = q_ij^T A q_ij with q_ij = a_i o a_j, for j in N(i). */
    i64 T = 0;
    for (i64 x = 0; x < di; x++) {
        i64 j = Ni[x];
        i64 nq = intersect(Ni, di, g->ci + g->rp[j], deg(g, j), q, qpos);
        /* q^T A q = sum over k, l in supp(q) of A(k,l) */
        for (i64 s = 0; s < nq; s++) {
            i64 k = q[s];
            const i32* Nk = g->ci + g->rp[k];
            i64 dk = deg(g, k);
            i64 cnt = 0;
            /* count |supp(q) ∩ N(k)|: merge when the lists are of similar size,
             * binary search of q in N(k) when N(k) is much longer */
            if (dk > 8 * nq) {
                for (i64 s2 = 0; s2 < nq; s2++) cnt += find_pos(Nk, dk, (i32)q[s2]) >= 0;
            } else {
                i64 u = 0, w = 0;
                while (u < nq && w < dk) {
                    if (q[u] < Nk[w]) u++;
                    else if (q[u] > Nk[w]) w++;
                    else { cnt++; u++; w++; }
                }
            }
            T += cnt;
        }
    }
    r.T = T; /* row sum of T; divided by 6 by the caller */
    return r;
}

/* ---------------------------------------------------------------------------
 * Step 8: net = U16^{-1} raw, by back substitution of U16 net = raw (Table II).
 * ------------------------------------------------------------------------- */
static void raw_to_net_row(const i64* raw, i64* net) {
    for (int k = NG - 1; k >= 0; k--) {
        i64 s = raw[k];
        for (int l = k + 1; l < NG; l++) s -= U16[k][l] * net[l];
        net[k] = s; /* U16[k][k] == 1 */
    }
}

void oracle_raw_to_net(i64 n, const i64* raw, i64* net) {
    for (i64 v = 0; v < n; v++) raw_to_net_row(raw + NG * v, net + NG * v);
}

/* Sub-dictionary with index set s = cols[0..k) (increasing): the conversion
 * matrix is U16(s,s) (Table II caption), so net(s) solves U16(s,s) net = raw(s),
 * by back substitution. raw and net are [n][k]. */
void oracle_raw_to_net_sub(i64 n, int k, const int* cols, const i64* raw, i64* net) {
    for (i64 v = 0; v < n; v++) {
        const i64* r = raw + (i64)k * v;
        i64* f = net + (i64)k * v;
        for (int a = k - 1; a >= 0; a--) {
            i64 s = r[a];
            for (int b = a + 1; b < k; b++) s -= U16[cols[a]][cols[b]] * f[b];
            f[a] = s; /* U16[cols[a]][cols[a]] == 1 */
        }
    }
}

/* ---------------------------------------------------------------------------
 * Driver. verts == NULL: all vertices, rows written in vertex order.
 * Otherwise rows for verts[0..nv) in that order. The rows of Table I at a
 * vertex i read C3 on the edges of i and of its neighbours (c3 at the
 * neighbours, the C3(j,k) of D4,c), so C3 and c3 are then computed only on the
 * rows of the closed neighbourhoods of the requested vertices, and p3 only at
 * the requested vertices; every value the requested rows read is the same as
 * in the full computation.
 * t_c3 (nullable, [n]) receives the seconds step 2 spent on each row it
 * computed; t_row (nullable, [rows]) the seconds steps 4-8 spent on each
 * output row. They are measurements only and change no result.
 * Returns 0 on success, -1 on allocation failure.
 * ------------------------------------------------------------------------- */
int oracle_fglt_timed(i64 n, const i64* rowptr, const i32* colidx, const i64* verts, i64 nv,
                      i64* raw, i64* net, int nthreads, double* t_c3, double* t_row) {
    graph G = {n, rowptr, colidx};
    const graph* g = &G;
    if (nthreads <= 0) {
#ifdef _OPENMP
        nthreads = omp_get_max_threads();
#else
        nthreads = 1;
#endif
    }
    i64 nnz = rowptr[n];
    i64* p1 = (i64*)malloc(sizeof(i64) * (n ? n : 1));
    i64* p2 = (i64*)malloc(sizeof(i64) * (n ? n : 1));
    i64* c3 = (i64*)malloc(sizeof(i64) * (n ? n : 1));
    i64* p3 = (i64*)malloc(sizeof(i64) * (n ? n : 1));
    i64* C3 = (i64*)calloc((size_t)(nnz ? nnz : 1), sizeof(i64));
    unsigned char* need = verts ? (unsigned char*)calloc((size_t)(n ? n : 1), 1) : NULL;
    if (!p1 || !p2 || !c3 || !p3 || !C3 || (verts && !need)) {
        free(p1); free(p2); free(c3); free(p3); free(C3); free(need);
        return -1;
    }
    if (verts) {
        for (i64 r = 0; r < nv; r++) {
            i64 i = verts[r];
            need[i] = 2; /* requested row */
            for (i64 e = rowptr[i]; e < rowptr[i + 1]; e++)
                if (!need[colidx[e]]) need[colidx[e]] = 1;
        }
    }

    /* Step 1: p1 = A e (= d1), p2 = A p1 - c2, c2 = d1. */
    for (i64 i = 0; i < n; i++) p1[i] = deg(g, i);
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (i64 i = 0; i < n; i++) {
        i64 s = 0;
        for (i64 e = rowptr[i]; e < rowptr[i + 1]; e++) s += p1[colidx[e]];
        p2[i] = rsub(s, p1[i]);
    }

    /* Step 2: C3 and c3 = C3 e / 2. */
    step_C3(g, C3, need, nthreads, t_c3);
    for (i64 i = 0; i < n; i++) {
        if (need && !need[i]) { c3[i] = 0; continue; }
        i64 s = 0;
        for (i64 e = rowptr[i]; e < rowptr[i + 1]; e++) s += C3[e];
        c3[i] = s / 2;
    }

    /* Step 3: p3 = A p2 - p1 o (p1 - 1) - 2 c3. */
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (i64 i = 0; i < n; i++) {
        if (need && need[i] != 2) { p3[i] = 0; continue; }
        i64 s = 0;
        for (i64 e = rowptr[i]; e < rowptr[i + 1]; e++) s += p2[colidx[e]];
        p3[i] = rsub(rsub(s, p1[i] * rsub(p1[i], 1)), 2 * c3[i]);
    }

    i64 rows = verts ? nv : n;
    int failed = 0;
#pragma omp parallel num_threads(nthreads)
    {
        i64* acc = (i64*)calloc((size_t)(n ? n : 1), sizeof(i64));
        i64* touched = (i64*)malloc(sizeof(i64) * (n ? 2 * n : 1));
        if (!acc || !touched) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (i64 r = 0; r < rows; r++) {
                const double t0 = t_row ? wall_s() : 0.0;
                i64 i = verts ? verts[r] : r;
                i64 d = p1[i];
                i64* f = raw + NG * r;
                /* Step 4: Table I rows built from vectors and SpMVs. */
                i64 Ap1m = 0, Ac3 = 0, C3p1m2 = 0;
                for (i64 e = rowptr[i]; e < rowptr[i + 1]; e++) {
                    i64 j = colidx[e];
                    Ap1m += rsub(p1[j], 1) * rsub(p1[j], 2); /* A((p1-1) o (p1-2)) */
                    Ac3 += c3[j];                           /* A c3 */
                    C3p1m2 += C3[e] * rsub(p1[j], 2);       /* C3 (p1 - 2) */
                }
                f[0] = 1;                                            /* e */
                f[1] = d;                                            /* p1 */
                f[2] = p2[i];                                        /* p2 */
                f[3] = d * rsub(d, 1) / 2;                           /* p1 o (p1-1) / 2 */
                f[4] = c3[i];                                        /* c3 */
                f[5] = p3[i];                                        /* p3 */
                f[6] = rsub(p2[i] * rsub(d, 1), 2 * c3[i]);          /* p2 o (p1-1) - 2 c3 */
                f[7] = Ap1m / 2;                                     /* A((p1-1)o(p1-2))/2 */
                f[8] = (d * rsub(d, 1) / 2) * rsub(d, 2) / 3;        /* p1(p1-1)(p1-2)/6 */
                f[9] = rsub(Ac3, 2 * c3[i]);                         /* A c3 - 2 c3 */
                f[10] = C3p1m2;                                      /* C3 (p1 - 2) */
                f[11] = rsub(d, 2) * c3[i];                          /* (p1 - 2) o c3 */
                /* Steps 5-7. */
                quad_terms qt = quad_row(g, i, C3, acc, touched);
                f[12] = qt.c4;                                       /* c4 = C4,2 e / 2 */
                f[13] = qt.d4c / 2;                                  /* D4,c e / 2 */
                f[14] = qt.d43 / 2;                                  /* D4,3 e / 2 */
                f[15] = qt.T / 6;                                    /* T e / 6 */
                if (net) raw_to_net_row(f, net + NG * r);
                if (t_row) t_row[r] = wall_s() - t0;
            }
        }
        free(acc);
        free(touched);
    }
    free(p1); free(p2); free(c3); free(p3); free(C3); free(need);
    return failed ? -1 : 0;
}

int oracle_fglt(i64 n, const i64* rowptr, const i32* colidx, const i64* verts, i64 nv,
                i64* raw, i64* net, int nthreads) {
    return oracle_fglt_timed(n, rowptr, colidx, verts, nv, raw, net, nthreads, NULL, NULL);
}

/* Number of threads an OpenMP region would use (for reporting). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
