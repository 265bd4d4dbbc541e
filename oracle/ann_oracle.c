/*
 * Plain CPU oracle for the divide-and-merge graph-index build of ScaleGANN
 * (arxiv 2605.10135).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the CPU-baseline leg of the benchmark call it; the library never does.
 *
 * Everything here is a direct, slow restatement of the definitions: no
 * blocking, no fusion, no reordering of sums beyond the plain loop order.  It
 * shares no code, header or constant with the CUDA library.
 *
 * Precision.  Reported distances are FP64 sums of squared differences (the
 * plain definition).  Where a floating-point value decides an integer (the
 * nearest k-means centroid, the r nearest shards, the beam-search frontier)
 * the decision is taken in FP32 with the sum evaluated term by term in index
 * order, without fused multiply-add ("d32"), which is the precision the GPU
 * kernels take the same decision in; FP64 sums of the k-means centroids follow
 * the sample order.  Built with -ffp-contract=off so the compiler cannot fuse.
 *
 * Element types: 0 = float32, 1 = float16, 2 = bfloat16, 3 = uint8.
 *
 * Parity status: every function below is pinned by the CPU tests (brute force,
 * hand-worked examples, library routines, invariants); none is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PAD 0xFFFFFFFFu

/* ---- element access: exact conversion of one stored element ---------- */

static float half_to_float(uint16_t h) {
    uint32_t sign = (uint32_t)(h >> 15) << 31;
    uint32_t e = (h >> 10) & 0x1f, m = h & 0x3ff, bits;
    if (e == 0) {
        if (m == 0) {
            bits = sign;
        } else { /* subnormal: normalise */
            int sh = 0;
            while (!(m & 0x400)) { m <<= 1; sh++; }
            m &= 0x3ff;
            bits = sign | ((uint32_t)(127 - 15 - sh + 1) << 23) | (m << 13);
        }
    } else if (e == 31) {
        bits = sign | 0x7f800000u | (m << 13);
    } else {
        bits = sign | ((e - 15 + 127) << 23) | (m << 13);
    }
    float f;
    memcpy(&f, &bits, 4);
    return f;
}

static float elem_f(const void* X, int dtype, int64_t i) {
    switch (dtype) {
    case 0: return ((const float*)X)[i];
    case 1: return half_to_float(((const uint16_t*)X)[i]);
    case 2: {
        uint32_t b = (uint32_t)((const uint16_t*)X)[i] << 16;
        float f;
        memcpy(&f, &b, 4);
        return f;
    }
    default: return (float)((const uint8_t*)X)[i];
    }
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- distances ------------------------------------------------------- */

/* Squared Euclidean distance in FP64, the plain definition. */
double or_d64(const void* X, int dtype, int64_t a, const void* Y, int ydtype, int64_t b, int d) {
    double s = 0.0;
    for (int t = 0; t < d; t++) {
        double df = (double)elem_f(X, dtype, a * d + t) - (double)elem_f(Y, ydtype, b * d + t);
        s += df * df;
    }
    return s;
}

/* Squared Euclidean distance in FP32, terms added in index order, unfused. */
float or_d32(const void* X, int dtype, int64_t a, const void* Y, int ydtype, int64_t b, int d) {
    float s = 0.0f;
    for (int t = 0; t < d; t++) {
        float df = elem_f(X, dtype, a * d + t) - elem_f(Y, ydtype, b * d + t);
        float sq = df * df;
        s = s + sq;
    }
    return s;
}

/* ---- k-means (Sec. IV Workflow step 1; Sec. II-B: shards by k-means) ----
 * Lloyd iterations on a sample: assign every sample point to the nearest
 * centroid by (d32, centroid id); each centroid becomes the FP64 mean of its
 * points (sums taken in sample order), rounded to float; an empty cluster
 * keeps its previous centroid. */
void or_kmeans(const void* X, int64_t N, int d, int dtype, int C, const float* init,
               const uint32_t* sample_idx, int64_t S, int iters, float* cent_out,
               int32_t* labels_out) {
    (void)N;
    memcpy(cent_out, init, sizeof(float) * (size_t)C * d);
    int32_t* lab = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S > 0 ? S : 1));
    double* sums = (double*)malloc(sizeof(double) * (size_t)C * d);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)C);
    for (int it = 0; it < iters; it++) {
        #pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < S; s++) {
            int best = 0;
            float bd = or_d32(X, dtype, sample_idx[s], cent_out, 0, 0, d);
            for (int c = 1; c < C; c++) {
                float dc = or_d32(X, dtype, sample_idx[s], cent_out, 0, c, d);
                if (dc < bd) { bd = dc; best = c; }
            }
            lab[s] = best;
        }
        memset(sums, 0, sizeof(double) * (size_t)C * d);
        memset(cnt, 0, sizeof(int64_t) * (size_t)C);
        for (int64_t s = 0; s < S; s++) {
            int c = lab[s];
            cnt[c] += 1;
            for (int t = 0; t < d; t++)
                sums[(size_t)c * d + t] += (double)elem_f(X, dtype, (int64_t)sample_idx[s] * d + t);
        }
        for (int c = 0; c < C; c++) {
            if (cnt[c] == 0) continue;
            for (int t = 0; t < d; t++)
                cent_out[(size_t)c * d + t] = (float)(sums[(size_t)c * d + t] / (double)cnt[c]);
        }
    }
    if (labels_out) memcpy(labels_out, lab, sizeof(int32_t) * (size_t)S);
    free(lab); free(sums); free(cnt);
}

/* ---- replicated assignment (Sec. II-B: each vector in its r nearest
 * shards, "typically two"; Sec. VI-B2: one replication) ----------------
 * For every vector the r centroids that come first in the order
 * (d32(x, c), c).  use_d64 != 0 takes the decision on FP64 distances
 * instead (used only to pin the FP32 decision against the exact one). */
void or_assign(const void* X, int64_t N, int d, int dtype, const float* cent, int C, int r,
               int use_d64, uint32_t* assign_out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        double* dist = (double*)malloc(sizeof(double) * (size_t)C);
        char* taken = (char*)calloc((size_t)C, 1);
        for (int c = 0; c < C; c++)
            dist[c] = use_d64 ? or_d64(X, dtype, i, cent, 0, c, d)
                              : (double)or_d32(X, dtype, i, cent, 0, c, d);
        for (int q = 0; q < r; q++) {
            int best = -1;
            for (int c = 0; c < C; c++) {
                if (taken[c]) continue;
                if (best < 0 || dist[c] < dist[best]) best = c;
            }
            taken[best] = 1;
            assign_out[i * r + q] = (uint32_t)best;
        }
        free(dist); free(taken);
    }
}

/* Shard member lists: shard c holds the ids of every vector assigned to it,
 * in increasing id order (Sec. V-C: merging needs the original vector order). */
void or_shards(const uint32_t* assign, int64_t N, int r, int C, uint32_t* members,
               int64_t* offsets) {
    /* OR_PAD entries (a vector held by fewer than r shards, Sec. V-B) are skipped. */
    int64_t* fill = (int64_t*)calloc((size_t)C + 1, sizeof(int64_t));
    for (int64_t i = 0; i < N * r; i++)
        if (assign[i] != OR_PAD) fill[assign[i] + 1]++;
    offsets[0] = 0;
    for (int c = 0; c < C; c++) offsets[c + 1] = offsets[c] + fill[c + 1];
    for (int c = 0; c < C; c++) fill[c] = offsets[c];
    for (int64_t g = 0; g < N; g++)
        for (int q = 0; q < r; q++)
            if (assign[g * r + q] != OR_PAD) members[fill[assign[g * r + q]]++] = (uint32_t)g;
    free(fill);
}

/* ---- blockwise-adaptive assignment with selective replication (Sec. V-A,
 * Sec. V-B, Algorithm 1) -------------------------------------------------
 * Vectors are read once, in id order, in blocks of `block` vectors.  Per
 * vector v, its candidate centroids are the M first in the order (d32(v, c), c)
 * (M = C considers every centroid).  State per cluster c: tot (members so far),
 * org (originals so far), rep (replicas so far), rad2 (largest d32 of its
 * originals so far: the squared radius).
 *
 * For block b (1-based), in this order (Sec. V-A):
 *  1. originals: each v of the block, in id order, goes to its nearest
 *     available candidate, i.e. the first one with tot < cap (cap = 0: no
 *     limit); if none of the M has room it goes to its nearest one anyway and
 *     is counted as an overflow;
 *  2. statistics: rad2 takes the block's originals in; the replica threshold
 *     theta_c = max(0, cap - ceil(org_c * N / processed)) leaves room for the
 *     originals still to come, extrapolated from the rate seen so far
 *     (processed = vectors in blocks 1..b); cap = 0: no threshold;
 *  3. replicas (Algorithm 1): each v of the block, in id order, walks its
 *     candidates in order; with its original c at distance dd (squared), a
 *     candidate c' != c at squared distance dd' is taken while v is in fewer
 *     than omega shards, if rep_c' < theta_c' and tot_c' < cap (size check) and
 *        dd' < (eps * eps) * dd                      (distance constraint)
 *        dd' < ((eps * tau) * (eps * tau)) * rad2_c'  (radius constraint),
 *     tau = 1 + (tau0 - 1) / b; these are the paper's d' < eps d and
 *     d' < eps tau R[c'] on squared distances, evaluated in FP64 on the d32
 *     values exactly as written.  An infinite eps skips both constraints.
 *
 * assign_out [N x omega]: the original first, then replicas in candidate
 * order, then OR_PAD.  stats_out[0] = replicas, stats_out[1] = overflows. */
void or_selective(const void* X, int64_t N, int d, int dtype, const float* cent, int C,
                  int omega, int M, double eps, double tau0, int64_t block, int64_t cap,
                  uint32_t* assign_out, int64_t* stats_out) {
    uint32_t* cand = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(N > 0 ? N : 1) * M);
    float* cdd = (float*)malloc(sizeof(float) * (size_t)(N > 0 ? N : 1) * M);
    /* candidate lists: the M first centroids in (d32, id) order */
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; v++) {
        float* dist = (float*)malloc(sizeof(float) * (size_t)C);
        char* taken = (char*)calloc((size_t)C, 1);
        for (int c = 0; c < C; c++) dist[c] = or_d32(X, dtype, v, cent, 0, c, d);
        for (int j = 0; j < M; j++) {
            int best = -1;
            for (int c = 0; c < C; c++) {
                if (taken[c]) continue;
                if (best < 0 || dist[c] < dist[best]) best = c;
            }
            taken[best] = 1;
            cand[v * M + j] = (uint32_t)best;
            cdd[v * M + j] = dist[best];
        }
        free(dist); free(taken);
    }
    int64_t* tot = (int64_t*)calloc((size_t)C, sizeof(int64_t));
    int64_t* org = (int64_t*)calloc((size_t)C, sizeof(int64_t));
    int64_t* rep = (int64_t*)calloc((size_t)C, sizeof(int64_t));
    int64_t* theta = (int64_t*)calloc((size_t)C, sizeof(int64_t));
    float* rad2 = (float*)calloc((size_t)C, sizeof(float));
    int* orig_j = (int*)malloc(sizeof(int) * (size_t)(block > 0 ? block : 1));
    const int test = !isinf(eps);
    int64_t nrep = 0, novf = 0;
    for (int64_t i = 0; i < N * omega; i++) assign_out[i] = OR_PAD;
    for (int64_t b0 = 0, beta = 1; b0 < N; b0 += block, beta++) {
        const int64_t b1 = N - b0 < block ? N : b0 + block;
        /* 1. originals */
        for (int64_t v = b0; v < b1; v++) {
            int jj = -1;
            for (int j = 0; j < M; j++)
                if (cap == 0 || tot[cand[v * M + j]] < cap) { jj = j; break; }
            if (jj < 0) { jj = 0; novf++; }
            const uint32_t c = cand[v * M + jj];
            orig_j[v - b0] = jj;
            assign_out[v * omega] = c;
            tot[c]++;
            org[c]++;
            if (cdd[v * M + jj] > rad2[c]) rad2[c] = cdd[v * M + jj];
        }
        /* 2. thresholds */
        for (int c = 0; c < C; c++) {
            if (cap == 0) continue;
            const int64_t proj = (org[c] * N + b1 - 1) / b1;
            theta[c] = cap - proj > 0 ? cap - proj : 0;
        }
        const double tau = 1.0 + (tau0 - 1.0) / (double)beta;
        const double e2 = eps * eps, et = eps * tau, et2 = et * et;
        /* 3. replicas */
        for (int64_t v = b0; v < b1; v++) {
            const int jo = orig_j[v - b0];
            const uint32_t c = cand[v * M + jo];
            const double dd = (double)cdd[v * M + jo];
            int assigned = 1;
            for (int j = 0; j < M; j++) {
                if (assigned >= omega) break;
                const uint32_t c2 = cand[v * M + j];
                if (c2 == c) continue;
                if (cap != 0 && (rep[c2] >= theta[c2] || tot[c2] >= cap)) continue;
                const double dd2 = (double)cdd[v * M + j];
                if (test && !(dd2 < e2 * dd && dd2 < et2 * (double)rad2[c2])) continue;
                assign_out[v * omega + assigned] = c2;
                assigned++;
                rep[c2]++;
                tot[c2]++;
                nrep++;
            }
        }
    }
    if (stats_out) { stats_out[0] = nrep; stats_out[1] = novf; }
    free(cand); free(cdd); free(tot); free(org); free(rep); free(theta); free(rad2); free(orig_j);
}

/* ---- exact per-shard kNN (Sec. IV Workflow step 2; the shard graph of
 * intermediate degree L, Sec. III) ----------------------------------------
 * For member p of its shard: the k other members with the smallest
 * (d64, global id), self excluded by id, duplicates kept; missing slots are
 * (OR_PAD, +inf).  rows[] lists the member positions to evaluate (all of
 * them when rows == NULL); shard_of_row gives each listed row's shard. */
static int64_t shard_of(const int64_t* offsets, int C, int64_t p) {
    int lo = 0, hi = C - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (offsets[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

void or_shard_knn_rows(const void* X, int d, int dtype, const uint32_t* members,
                       const int64_t* offsets, int C, int k, const int64_t* rows, int64_t nrows,
                       uint32_t* id_out, double* d_out) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < nrows; q++) {
        int64_t p = rows ? rows[q] : q;
        int64_t s = shard_of(offsets, C, p);
        uint32_t u = members[p];
        uint32_t* ids = id_out + q * k;
        double* ds = d_out + q * k;
        for (int j = 0; j < k; j++) { ids[j] = OR_PAD; ds[j] = INFINITY; }
        for (int64_t m = offsets[s]; m < offsets[s + 1]; m++) {
            uint32_t v = members[m];
            if (v == u) continue;
            double dv = or_d64(X, dtype, u, X, dtype, v, d);
            /* insert (dv, v) into the sorted list if it ranks within k */
            int pos = k;
            while (pos > 0 && (ds[pos - 1] > dv || (ds[pos - 1] == dv && ids[pos - 1] > v))) pos--;
            if (pos >= k) continue;
            for (int j = k - 1; j > pos; j--) { ids[j] = ids[j - 1]; ds[j] = ds[j - 1]; }
            ids[pos] = v;
            ds[pos] = dv;
        }
    }
}

/* ---- pruning L -> R (intermediate degree L to final degree R, Sec. III and
 * Sec. VI-B2).  The paper does not print the rule; the reading used here is
 * the rank-based detour count, defined on the lists alone:
 *   L_u = [v_0 .. v_{m-1}] (valid entries), pos_w(v) = index of v in L_w;
 *   c_j = #{ i < j : pos_{v_i}(v_j) < j };
 *   keep the R entries with the smallest (c_j, j), emitted in increasing j.
 * rule == 1 keeps the first R entries (plain truncation).  The list of a
 * neighbour w is w's list in the same shard. */
static int64_t row_in_shard(const uint32_t* members, int64_t lo, int64_t hi, uint32_t v) {
    /* member lists are sorted by id: binary search */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (members[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

void or_prune(const uint32_t* knn_id, const double* knn_d, const uint32_t* members,
              const int64_t* offsets, int C, int k, int R, int rule, uint32_t* pr_id,
              double* pr_d) {
    int64_t rows = offsets[C];
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < rows; p++) {
        int64_t s = shard_of(offsets, C, p);
        const uint32_t* L = knn_id + p * k;
        int m = 0;
        while (m < k && L[m] != OR_PAD) m++;
        int* cnt = (int*)calloc((size_t)k, sizeof(int));
        char* keep = (char*)calloc((size_t)k, 1);
        if (rule == 0) {
            for (int j = 0; j < m; j++) {
                for (int i = 0; i < j; i++) {
                    int64_t w = row_in_shard(members, offsets[s], offsets[s + 1], L[i]);
                    const uint32_t* Lw = knn_id + w * k;
                    int pos = -1;
                    for (int t = 0; t < k; t++)
                        if (Lw[t] == L[j]) { pos = t; break; }
                    if (pos >= 0 && pos < j) cnt[j]++;
                }
            }
            /* choose R entries by (c_j, j) */
            int chosen = 0;
            while (chosen < R && chosen < m) {
                int best = -1;
                for (int j = 0; j < m; j++) {
                    if (keep[j]) continue;
                    if (best < 0 || cnt[j] < cnt[best]) best = j;
                }
                keep[best] = 1;
                chosen++;
            }
        } else {
            for (int j = 0; j < m && j < R; j++) keep[j] = 1;
        }
        int o = 0;
        for (int j = 0; j < m; j++) {
            if (!keep[j]) continue;
            pr_id[p * R + o] = L[j];
            pr_d[p * R + o] = knn_d[p * k + j];
            o++;
        }
        for (; o < R; o++) { pr_id[p * R + o] = OR_PAD; pr_d[p * R + o] = INFINITY; }
        free(cnt); free(keep);
    }
}

/* ---- merge by edge union (Sec. II-B; Sec. IV Workflow step 3) ----------
 * For each global id g: the union of g's pruned lists over the shards that
 * hold g, duplicates removed by id (the smaller distance kept), then the R
 * smallest by (distance, id), sorted, padded with (OR_PAD, +inf).  gids[]
 * lists the ids to evaluate (all when NULL). */
void or_merge(const uint32_t* pr_id, const double* pr_d, const uint32_t* members,
              const int64_t* offsets, int C, int64_t N, int R, const int64_t* gids, int64_t ng,
              uint32_t* graph, double* gdist, uint32_t* degree) {
    int64_t rows = offsets[C];
    /* rows of each g, by one counting pass over the member lists */
    int64_t* start = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    for (int64_t p = 0; p < rows; p++) start[members[p] + 1]++;
    for (int64_t g = 0; g < N; g++) start[g + 1] += start[g];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    memcpy(fill, start, sizeof(int64_t) * (size_t)N);
    int64_t* rowlist = (int64_t*)malloc(sizeof(int64_t) * (size_t)(rows > 0 ? rows : 1));
    for (int64_t p = 0; p < rows; p++) rowlist[fill[members[p]]++] = p;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < ng; q++) {
        int64_t g = gids ? gids[q] : q;
        int64_t cap = (start[g + 1] - start[g]) * R;
        uint32_t* cid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(cap > 0 ? cap : 1));
        double* cd = (double*)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
        int64_t n = 0;
        for (int64_t a = start[g]; a < start[g + 1]; a++) {
            int64_t p = rowlist[a];
            for (int j = 0; j < R; j++) {
                uint32_t v = pr_id[p * R + j];
                if (v == OR_PAD) continue;
                double dv = pr_d[p * R + j];
                int64_t e = 0;
                while (e < n && cid[e] != v) e++;
                if (e < n) {
                    if (dv < cd[e]) cd[e] = dv;
                } else {
                    cid[n] = v; cd[n] = dv; n++;
                }
            }
        }
        /* R smallest by (distance, id) by repeated selection */
        uint32_t* go = graph + q * R;
        double* gd = gdist + q * R;
        char* used = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
        int o = 0;
        for (; o < R && o < n; o++) {
            int64_t best = -1;
            for (int64_t e = 0; e < n; e++) {
                if (used[e]) continue;
                if (best < 0 || cd[e] < cd[best] || (cd[e] == cd[best] && cid[e] < cid[best])) best = e;
            }
            used[best] = 1;
            go[o] = cid[best];
            gd[o] = cd[best];
        }
        degree[q] = (uint32_t)o;
        for (; o < R; o++) { go[o] = OR_PAD; gd[o] = INFINITY; }
        free(cid); free(cd); free(used);
    }
    free(start); free(fill); free(rowlist);
}

/* ---- prune and merge variants (alternatives to the rank-detour prune and the
 * plain edge union; not printed in the paper, which inherits its prune from the
 * shard builder) ---------------------------------------------------------
 * Occlusion prune (the robust prune of graph builders in the Vamana family): walk
 * u's list in (distance, id) order and keep v unless some kept w satisfies
 * alpha * |w - v| <= |u - v|, i.e. on squared distances
 * (alpha * alpha) * d64(w, v) <= d64(u, v), where d64(u, v) is the distance the
 * list carries; stop at R kept.  Kept entries stay in list order. */
void or_prune_alpha(const void* X, int d, int dtype, const uint32_t* knn_id, const double* knn_d,
                    const uint32_t* members, int64_t rows, int k, int R, double alpha,
                    uint32_t* pr_id, double* pr_d) {
    const double a2 = alpha * alpha;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < rows; p++) {
        (void)members;
        int kept = 0;
        for (int j = 0; j < k && kept < R; j++) {
            const uint32_t v = knn_id[p * k + j];
            if (v == OR_PAD) continue;
            const double duv = knn_d[p * k + j];
            int occluded = 0;
            for (int e = 0; e < kept && !occluded; e++) {
                const uint32_t w = pr_id[p * R + e];
                if (a2 * or_d64(X, dtype, w, X, dtype, v, d) <= duv) occluded = 1;
            }
            if (occluded) continue;
            pr_id[p * R + kept] = v;
            pr_d[p * R + kept] = duv;
            kept++;
        }
        for (int e = kept; e < R; e++) {
            pr_id[p * R + e] = OR_PAD;
            pr_d[p * R + e] = INFINITY;
        }
    }
}

/* Merged graph with reverse edges: for every v, the first ceil(R/2) entries of its
 * list, then the vectors u whose lists hold v (each with the distance of that
 * edge) in (distance, id) order, then the rest of v's own list, skipping ids
 * already taken, up to R; the result sorted by (distance, id). */
void or_merge_reverse(const uint32_t* graph, const double* gdist, const uint32_t* degree,
                      int64_t N, int R, uint32_t* out_g, double* out_d, uint32_t* out_deg) {
    int64_t* cnt = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    for (int64_t u = 0; u < N; u++)
        for (uint32_t j = 0; j < degree[u]; j++) cnt[graph[u * R + j] + 1]++;
    for (int64_t v = 0; v < N; v++) cnt[v + 1] += cnt[v];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)N);
    const int64_t ne = cnt[N];
    uint32_t* rsrc = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(ne > 0 ? ne : 1));
    double* rdist = (double*)malloc(sizeof(double) * (size_t)(ne > 0 ? ne : 1));
    for (int64_t u = 0; u < N; u++)
        for (uint32_t j = 0; j < degree[u]; j++) {
            const uint32_t v = graph[u * R + j];
            rsrc[fill[v]] = (uint32_t)u;
            rdist[fill[v]] = gdist[u * R + j];
            fill[v]++;
        }
    const int half = (R + 1) / 2;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t v = 0; v < N; v++) {
        uint32_t* lid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)R);
        double* ld = (double*)malloc(sizeof(double) * (size_t)R);
        int n = 0;
        const int dv = (int)degree[v];
        for (int j = 0; j < dv && j < half; j++) {
            lid[n] = graph[v * R + j];
            ld[n] = gdist[v * R + j];
            n++;
        }
        /* reverse sources of v by (distance, id): repeated selection */
        const int64_t r0 = cnt[v], r1 = cnt[v + 1];
        char* used = (char*)calloc((size_t)(r1 - r0 + 1), 1);
        while (n < R) {
            int64_t best = -1;
            for (int64_t e = r0; e < r1; e++) {
                if (used[e - r0]) continue;
                if (best < 0 || rdist[e] < rdist[best] ||
                    (rdist[e] == rdist[best] && rsrc[e] < rsrc[best]))
                    best = e;
            }
            if (best < 0) break;
            used[best - r0] = 1;
            int dup = 0;
            for (int q = 0; q < n; q++) dup |= lid[q] == rsrc[best];
            if (dup) continue;
            lid[n] = rsrc[best];
            ld[n] = rdist[best];
            n++;
        }
        for (int j = half; j < dv && n < R; j++) {
            int dup = 0;
            for (int q = 0; q < n; q++) dup |= lid[q] == graph[v * R + j];
            if (dup) continue;
            lid[n] = graph[v * R + j];
            ld[n] = gdist[v * R + j];
            n++;
        }
        /* sorted by (distance, id) */
        for (int a = 1; a < n; a++)
            for (int b = a; b > 0 && (ld[b] < ld[b - 1] || (ld[b] == ld[b - 1] && lid[b] < lid[b - 1])); b--) {
                const uint32_t ti = lid[b]; lid[b] = lid[b - 1]; lid[b - 1] = ti;
                const double td = ld[b]; ld[b] = ld[b - 1]; ld[b - 1] = td;
            }
        for (int q = 0; q < R; q++) {
            out_g[v * R + q] = q < n ? lid[q] : OR_PAD;
            out_d[v * R + q] = q < n ? ld[q] : INFINITY;
        }
        out_deg[v] = (uint32_t)n;
        free(lid); free(ld); free(used);
    }
    free(cnt); free(fill); free(rsrc); free(rdist);
}

/* ---- query evaluation (Sec. VI-B2: a CPU query following DiskANN's search
 * strategy; top-10 recall) ---------------------------------------------
 * Medoid: the vector nearest (d32) to the FP64 mean rounded to float, ties to
 * the smaller id. */
int64_t or_medoid(const void* X, int64_t N, int d, int dtype) {
    double* mean = (double*)calloc((size_t)d, sizeof(double));
    float* mf = (float*)malloc(sizeof(float) * (size_t)d);
    for (int64_t i = 0; i < N; i++)
        for (int t = 0; t < d; t++) mean[t] += (double)elem_f(X, dtype, i * d + t);
    for (int t = 0; t < d; t++) mf[t] = (float)(mean[t] / (double)N);
    int64_t best = 0;
    float bd = or_d32(X, dtype, 0, mf, 0, 0, d);
    for (int64_t i = 1; i < N; i++) {
        float di = or_d32(X, dtype, i, mf, 0, 0, d);
        if (di < bd) { bd = di; best = i; }
    }
    free(mean); free(mf);
    return best;
}

/* Best-first beam search with list size Ls: start at the entry vertex; take
 * the closest unexpanded entry of the list, expand it (each out-neighbour not
 * yet seen is marked seen, its d32 distance computed and inserted if it ranks
 * within Ls by (distance, id)); stop when every listed entry is expanded.
 * Returns the first topk ids and, per query, the number of distances computed. */
void or_search(const uint32_t* graph, const uint32_t* degree, int R, const void* X, int64_t N,
               int d, int dtype, const void* Q, int qdtype, int64_t nq, int64_t entry, int Ls,
               int topk, uint32_t* out_ids, int64_t* out_count) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nq; q++) {
        char* seen = (char*)calloc((size_t)N, 1);
        uint32_t* lid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)Ls);
        float* ld = (float*)malloc(sizeof(float) * (size_t)Ls);
        char* lexp = (char*)malloc((size_t)Ls);
        int n = 1;
        int64_t count = 1;
        lid[0] = (uint32_t)entry;
        ld[0] = or_d32(Q, qdtype, q, X, dtype, entry, d);
        lexp[0] = 0;
        seen[entry] = 1;
        for (;;) {
            int cur = -1;
            for (int e = 0; e < n; e++)
                if (!lexp[e]) { cur = e; break; }
            if (cur < 0) break;
            lexp[cur] = 1;
            uint32_t u = lid[cur];
            for (uint32_t j = 0; j < degree[u]; j++) {
                uint32_t v = graph[(int64_t)u * R + j];
                if (v == OR_PAD || seen[v]) continue;
                seen[v] = 1;
                float dv = or_d32(Q, qdtype, q, X, dtype, v, d);
                count++;
                int pos = n;
                while (pos > 0 && (ld[pos - 1] > dv || (ld[pos - 1] == dv && lid[pos - 1] > v))) pos--;
                if (pos >= Ls) continue;
                int last = n < Ls ? n : Ls - 1;
                for (int e = last; e > pos; e--) { lid[e] = lid[e - 1]; ld[e] = ld[e - 1]; lexp[e] = lexp[e - 1]; }
                lid[pos] = v; ld[pos] = dv; lexp[pos] = 0;
                if (n < Ls) n++;
            }
        }
        for (int e = 0; e < topk; e++) out_ids[q * topk + e] = e < n ? lid[e] : OR_PAD;
        out_count[q] = count;
        free(seen); free(lid); free(ld); free(lexp);
    }
}

/* Exact top-k of every query over all N vectors by (d64, id): the ground
 * truth of the recall measurement. */
void or_bruteforce(const void* X, int64_t N, int d, int dtype, const void* Q, int qdtype,
                   int64_t nq, int k, uint32_t* id_out, double* d_out) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; q++) {
        uint32_t* ids = id_out + q * k;
        double* ds = d_out + q * k;
        for (int j = 0; j < k; j++) { ids[j] = OR_PAD; ds[j] = INFINITY; }
        for (int64_t v = 0; v < N; v++) {
            double dv = or_d64(Q, qdtype, q, X, dtype, v, d);
            int pos = k;
            while (pos > 0 && (ds[pos - 1] > dv || (ds[pos - 1] == dv && ids[pos - 1] > v))) pos--;
            if (pos >= k) continue;
            for (int j = k - 1; j > pos; j--) { ids[j] = ids[j - 1]; ds[j] = ds[j - 1]; }
            ids[pos] = (uint32_t)v;
            ds[pos] = dv;
        }
    }
}
