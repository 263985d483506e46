/*
 * efm_oracle.c -- plain, slow CPU oracle for the exhaustive flux-balanced
 * pathway traversal.  TEST INFRASTRUCTURE ONLY: the library never links,
 * loads or calls this file; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes (one job = one network, one target metabolite):
 *
 *  Network (Sec. 2.1, Def. 2): S is m x n; reversible reactions are split
 *  into a forward column followed by a reverse column (the "direction" of
 *  Def. 6), twin[] links the two.  S_int keeps the internal rows only, in
 *  original metabolite order; steady state is imposed on those rows.
 *
 *  Seeds (INIT kernel, Sec. 4.1; Def. 8; Prop. 1): for target t every
 *  column j with S[t][j] > 0 gives the pathway U = {j} with flux 1 on j,
 *  so its extra flux vector is EF = S_int[:, j] (Eq. 2).  t = -1 seeds
 *  every column.
 *
 *  A pathway state is (U, EF, sec): the support, the extra flux of every
 *  internal metabolite divided by the gcd of its entries (the flux vector
 *  is kept only as a ray, positive on U), and the count of secondary steps
 *  (Def. 10) taken so far.
 *
 *  Step (METAx, Alg. 3, restated deterministically and exhaustively):
 *  EF == 0 on every internal metabolite -> the pathway is balanced (all
 *  metabolites Stable, "Done").  Otherwise the acting metabolite i is the
 *  unbalanced one with the fewest reactions able to fix it (ties by index);
 *  EF_i > 0 is a forward flow (Def. 9) and every output reaction k of i
 *  (S_ik < 0) is tried, EF_i < 0 is a backward flow and every input reaction
 *  (S_ik > 0) is tried -- all OR branches instead of one random choice.
 *  The new flux on k zeroes EF_i (Eq. 3 in integers):
 *      g = gcd(|EF_i|, |S_ik|), a = |S_ik|/g, c = |EF_i|/g,
 *      EF' = a*EF + c*S_int[:, k],      then divided by gcd(EF').
 *  If k is already in U the step is secondary (Eq. 4: flux added on a
 *  reaction already in the pathway) and costs one unit of max_secondary
 *  (the MAX_LOOP bound of Sec. 3.2); otherwise it adds a column and
 *  |U| + 1 <= max_len must hold.  A column whose twin is in U is never
 *  taken.  A child whose EF' has an entry outside the int32 range is
 *  dropped and counted as overflow.
 *
 *  Arbiter (Sec. 3.2.2, Def. 3): a balanced support U is a result iff
 *  nullity over Q of S_int[:, U] is 1 (the flux ray is then the only
 *  balanced mode on U, so no balanced mode has a smaller support).  The
 *  rank is computed exactly (fraction-free Bareiss elimination).
 *
 *  Search (breadth first by level; level 0 = seeds; level l expands the
 *  frontier F_{l-1}):
 *    - a balanced support is judged once per job (a set of seen supports);
 *    - a non-balanced child whose new column k completes the support of a
 *      result accepted at a level < l (k in E, E contained in U + {k}) is
 *      pruned: any balanced descendant would contain that result, so it could
 *      not be minimal (secondary steps, k already in U, are never pruned).
 *      The rule is an optimisation, not part of the definition (Def. 3 only
 *      asks for nullity 1): with flags & OR_NO_PRUNE it is skipped, and the
 *      result set must not change (pinned by the tests);
 *    - F_l = distinct (U, EF) among the remaining children (equal keys at
 *      one level have equal sec);
 *    - if |F_l| > max_frontier (> 0): status TRUNCATED, stop; results of
 *      level l are kept, F_l is not counted;
 *    - if the result count >= max_results (> 0): status CAPPED, stop and
 *      return the max_results smallest;
 *    - stop when F_l is empty.
 *  Output: distinct supports sorted by (|U|, ascending column list).
 *
 *  Subtractive variant (flags & OR_SUBTRACTIVE; Eq. 5, Prop. 3): a state
 *  also carries its flux vector v (integers, positive on U; EF = S_int v),
 *  and (EF, v) are divided together by the gcd of all their entries, so a
 *  state is the ray of v.  Besides the additive branches above, the acting
 *  metabolite i may be balanced by taking flux away from a reaction k
 *  already in U that moves i the same way as its imbalance (S_ik > 0 for a
 *  surplus EF_i > 0, S_ik < 0 for a deficit): with g, a, c as in Eq. 3,
 *      v' = a v - c e_k,   EF' = a EF - c S_int[:, k],
 *  which zeroes EF_i (Eq. 5 in integers).  It keeps U, costs one secondary
 *  step, and is discarded when the new flux on k is zero (Prop. 3) or
 *  negative (the split columns carry non-negative flux); such children are
 *  counted in zero_flux.  Additive steps update v as v' = a v + c e_k.
 *  Distinct states are distinct (U, v).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2
#define OR_ERANGE -3

#define OR_TRUNCATED 1
#define OR_CAPPED 2
#define OR_OVERFLOW_DROPPED 4

/* or_limits.flags */
#define OR_NO_PRUNE 1    /* the plain definition: no superset rule */
#define OR_SUBTRACTIVE 2 /* Eq. 5 steps as well (states carry their flux vector) */

typedef struct {
    int32_t max_len;
    int32_t max_secondary;
    int64_t max_results;
    int64_t max_frontier;
    int32_t flags; /* OR_* bits above */
    int32_t reserved;
} or_limits;

typedef struct {
    int64_t levels;
    int64_t seeds;
    int64_t expansions;
    int64_t overflow;
    int64_t balanced;
    int64_t candidates;
    int64_t results;
    int64_t pruned;
    int64_t frontier;
    int64_t frontier_max;
    int64_t status;
    int64_t zero_flux; /* Eq. 5 children discarded: a reaction's flux reached 0 or below (Prop. 3) */
} or_counters;

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

static uint64_t gcd_u64(uint64_t a, uint64_t b)
{
    while (b) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static uint64_t abs_i64(int64_t x) { return x < 0 ? (uint64_t)0 - (uint64_t)x : (uint64_t)x; }

static int popcount_words(const uint64_t *u, int W)
{
    int c = 0;
    for (int w = 0; w < W; ++w) c += __builtin_popcountll(u[w]);
    return c;
}

static int bit_test(const uint64_t *u, int k) { return (int)((u[k >> 6] >> (k & 63)) & 1u); }

/* ------------------------------------------------------------------------ */
/* exact rank over Q                                                         */
/*                                                                           */
/* Bareiss fraction-free elimination: after each pivot step every entry is  */
/* a minor of the input, and the division by the previous pivot is exact.    */
/* First in __int128 with overflow checks; on overflow the same elimination */
/* is repeated with a small arbitrary-precision integer type.                */
/* ------------------------------------------------------------------------ */

typedef __int128 i128;

static int rank_i128(int rows, int cols, const int64_t *A, int *rank_out)
{
    i128 *M = (i128 *)malloc(sizeof(i128) * (size_t)(rows > 0 ? rows : 1) * (size_t)(cols > 0 ? cols : 1));
    if (!M) return OR_ENOMEM;
    for (int i = 0; i < rows * cols; ++i) M[i] = A[i];
    int r = 0;
    i128 prev = 1;
    for (int c = 0; c < cols && r < rows; ++c) {
        int piv = -1;
        for (int i = r; i < rows; ++i)
            if (M[i * cols + c] != 0) { piv = i; break; }
        if (piv < 0) continue;
        if (piv != r)
            for (int j = 0; j < cols; ++j) {
                i128 t = M[r * cols + j];
                M[r * cols + j] = M[piv * cols + j];
                M[piv * cols + j] = t;
            }
        i128 p = M[r * cols + c];
        for (int i = r + 1; i < rows; ++i) {
            i128 f = M[i * cols + c];
            for (int j = c + 1; j < cols; ++j) {
                i128 x, y, z;
                if (__builtin_mul_overflow(p, M[i * cols + j], &x) ||
                    __builtin_mul_overflow(f, M[r * cols + j], &y) ||
                    __builtin_sub_overflow(x, y, &z)) {
                    free(M);
                    return OR_ERANGE;
                }
                M[i * cols + j] = z / prev;
            }
            M[i * cols + c] = 0;
        }
        prev = p;
        ++r;
    }
    free(M);
    *rank_out = r;
    return OR_OK;
}

/* --- arbitrary precision signed integers (sign + magnitude, 32-bit limbs) */

typedef struct {
    int sign; /* -1, 0, +1 */
    int n;    /* used limbs */
    int cap;
    uint32_t *d;
} big;

static int big_reserve(big *a, int n)
{
    if (a->cap >= n) return 0;
    uint32_t *p = (uint32_t *)realloc(a->d, sizeof(uint32_t) * (size_t)n);
    if (!p) return -1;
    a->d = p;
    a->cap = n;
    return 0;
}

static void big_trim(big *a)
{
    while (a->n > 0 && a->d[a->n - 1] == 0) --a->n;
    if (a->n == 0) a->sign = 0;
}

static int big_set_i64(big *a, int64_t v)
{
    if (big_reserve(a, 2)) return -1;
    uint64_t m = abs_i64(v);
    a->d[0] = (uint32_t)m;
    a->d[1] = (uint32_t)(m >> 32);
    a->n = 2;
    a->sign = v < 0 ? -1 : 1;
    big_trim(a);
    return 0;
}

static int mag_cmp(const big *a, const big *b)
{
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int i = a->n - 1; i >= 0; --i)
        if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
    return 0;
}

/* r = |a| + |b| (magnitudes), r must not alias */
static int mag_add(big *r, const big *a, const big *b)
{
    int n = (a->n > b->n ? a->n : b->n) + 1;
    if (big_reserve(r, n)) return -1;
    uint64_t carry = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t s = carry;
        if (i < a->n) s += a->d[i];
        if (i < b->n) s += b->d[i];
        r->d[i] = (uint32_t)s;
        carry = s >> 32;
    }
    r->n = n;
    return 0;
}

/* r = |a| - |b| with |a| >= |b|, r must not alias */
static int mag_sub(big *r, const big *a, const big *b)
{
    if (big_reserve(r, a->n > 0 ? a->n : 1)) return -1;
    int64_t borrow = 0;
    for (int i = 0; i < a->n; ++i) {
        int64_t s = (int64_t)a->d[i] - borrow - (i < b->n ? (int64_t)b->d[i] : 0);
        borrow = s < 0;
        if (s < 0) s += ((int64_t)1 << 32);
        r->d[i] = (uint32_t)s;
    }
    r->n = a->n;
    return 0;
}

/* r = a - b */
static int big_sub(big *r, const big *a, const big *b)
{
    if (b->sign == 0) {
        if (big_reserve(r, a->n > 0 ? a->n : 1)) return -1;
        memcpy(r->d, a->d, sizeof(uint32_t) * (size_t)a->n);
        r->n = a->n;
        r->sign = a->sign;
        return 0;
    }
    if (a->sign == 0) {
        if (big_reserve(r, b->n)) return -1;
        memcpy(r->d, b->d, sizeof(uint32_t) * (size_t)b->n);
        r->n = b->n;
        r->sign = -b->sign;
        return 0;
    }
    if (a->sign != b->sign) { /* a - b = sign(a) * (|a| + |b|) */
        if (mag_add(r, a, b)) return -1;
        r->sign = a->sign;
    } else {
        int c = mag_cmp(a, b);
        if (c >= 0) {
            if (mag_sub(r, a, b)) return -1;
            r->sign = a->sign;
        } else {
            if (mag_sub(r, b, a)) return -1;
            r->sign = -a->sign;
        }
    }
    big_trim(r);
    return 0;
}

/* r = a * b, r must not alias */
static int big_mul(big *r, const big *a, const big *b)
{
    if (a->sign == 0 || b->sign == 0) {
        r->n = 0;
        r->sign = 0;
        return 0;
    }
    int n = a->n + b->n;
    if (big_reserve(r, n)) return -1;
    memset(r->d, 0, sizeof(uint32_t) * (size_t)n);
    for (int i = 0; i < a->n; ++i) {
        uint64_t carry = 0;
        for (int j = 0; j < b->n; ++j) {
            uint64_t t = (uint64_t)a->d[i] * b->d[j] + r->d[i + j] + carry;
            r->d[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        int k = i + b->n;
        while (carry) {
            uint64_t t = (uint64_t)r->d[k] + carry;
            r->d[k] = (uint32_t)t;
            carry = t >> 32;
            ++k;
        }
    }
    r->n = n;
    r->sign = a->sign * b->sign;
    big_trim(r);
    return 0;
}

/* q = a / b for an exact division, by binary long division on magnitudes */
static int big_divexact(big *q, const big *a, const big *b)
{
    if (a->sign == 0) {
        q->n = 0;
        q->sign = 0;
        return 0;
    }
    big rem = {0, 0, 0, NULL}, tmp = {0, 0, 0, NULL};
    int nbits = a->n * 32;
    if (a->n <= 0) return -1;
    if (big_reserve(q, a->n) || big_reserve(&rem, a->n + 1) || big_reserve(&tmp, a->n + 1)) goto fail;
    memset(q->d, 0, sizeof(uint32_t) * (size_t)a->n);
    q->n = a->n;
    rem.n = 0;
    rem.sign = 0;
    for (int bit = nbits - 1; bit >= 0; --bit) {
        /* rem = 2 * rem + bit */
        uint32_t carry = (a->d[bit >> 5] >> (bit & 31)) & 1u;
        for (int i = 0; i < rem.n; ++i) {
            uint32_t nc = rem.d[i] >> 31;
            rem.d[i] = (rem.d[i] << 1) | carry;
            carry = nc;
        }
        if (carry) rem.d[rem.n++] = carry;
        if (rem.n) rem.sign = 1;
        if (mag_cmp(&rem, b) >= 0) {
            if (mag_sub(&tmp, &rem, b)) goto fail;
            memcpy(rem.d, tmp.d, sizeof(uint32_t) * (size_t)tmp.n);
            rem.n = tmp.n;
            big_trim(&rem);
            q->d[bit >> 5] |= 1u << (bit & 31);
        }
    }
    q->sign = a->sign * b->sign;
    big_trim(q);
    free(rem.d);
    free(tmp.d);
    return 0;
fail:
    free(rem.d);
    free(tmp.d);
    return -1;
}

static int rank_big(int rows, int cols, const int64_t *A, int *rank_out)
{
    int total = rows * cols;
    big *M = (big *)calloc((size_t)(total > 0 ? total : 1), sizeof(big));
    big prev = {0, 0, 0, NULL}, x = {0, 0, 0, NULL}, y = {0, 0, 0, NULL}, z = {0, 0, 0, NULL};
    int rc = OR_ENOMEM;
    if (!M) return OR_ENOMEM;
    for (int i = 0; i < total; ++i)
        if (big_set_i64(&M[i], A[i])) goto done;
    if (big_set_i64(&prev, 1)) goto done;
    int r = 0;
    for (int c = 0; c < cols && r < rows; ++c) {
        int piv = -1;
        for (int i = r; i < rows; ++i)
            if (M[i * cols + c].sign != 0) { piv = i; break; }
        if (piv < 0) continue;
        if (piv != r)
            for (int j = 0; j < cols; ++j) {
                big t = M[r * cols + j];
                M[r * cols + j] = M[piv * cols + j];
                M[piv * cols + j] = t;
            }
        for (int i = r + 1; i < rows; ++i) {
            for (int j = c + 1; j < cols; ++j) {
                if (big_mul(&x, &M[r * cols + c], &M[i * cols + j])) goto done;
                if (big_mul(&y, &M[i * cols + c], &M[r * cols + j])) goto done;
                if (big_sub(&z, &x, &y)) goto done;
                if (big_divexact(&M[i * cols + j], &z, &prev)) goto done;
            }
            M[i * cols + c].sign = 0;
            M[i * cols + c].n = 0;
        }
        big *p = &M[r * cols + c];
        if (big_reserve(&prev, p->n > 0 ? p->n : 1)) goto done;
        memcpy(prev.d, p->d, sizeof(uint32_t) * (size_t)p->n);
        prev.n = p->n;
        prev.sign = p->sign;
        ++r;
    }
    *rank_out = r;
    rc = OR_OK;
done:
    for (int i = 0; i < total; ++i) free(M[i].d);
    free(M);
    free(prev.d);
    free(x.d);
    free(y.d);
    free(z.d);
    return rc;
}

/* Exact rank of a rows x cols integer matrix (row-major).  force_big = 1
 * skips the __int128 attempt (used by tests to exercise the fallback). */
int oracle_rank(int32_t rows, int32_t cols, const int64_t *A, int32_t force_big, int32_t *rank_out)
{
    int r = 0, rc;
    if (rows <= 0 || cols <= 0) {
        *rank_out = 0;
        return OR_OK;
    }
    if (!force_big) {
        rc = rank_i128(rows, cols, A, &r);
        if (rc == OR_OK) {
            *rank_out = r;
            return OR_OK;
        }
        if (rc != OR_ERANGE) return rc;
    }
    rc = rank_big(rows, cols, A, &r);
    if (rc == OR_OK) *rank_out = r;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* network normalisation                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n_met, n_rxn;
    int M;         /* internal metabolites */
    int N;         /* split columns */
    int W;         /* 64-bit words per support */
    int *int_row;  /* metabolite -> internal row or -1 */
    int *twin;     /* column -> twin column or -1 */
    int *col_rxn;  /* column -> original reaction */
    int *col_dir;  /* +1 forward, -1 reverse */
    int64_t *S;    /* S_int, M x N row-major */
    int *deg_out;  /* per internal row: #columns consuming it (S < 0) */
    int *deg_in;   /* per internal row: #columns producing it (S > 0) */
} or_net;

static void net_free(or_net *g)
{
    free(g->int_row);
    free(g->twin);
    free(g->col_rxn);
    free(g->col_dir);
    free(g->S);
    free(g->deg_out);
    free(g->deg_in);
}

static int net_build(or_net *g, int n_met, int n_rxn, const int32_t *row_ptr, const int32_t *col_idx,
                     const int32_t *coef, const uint8_t *reversible, const uint8_t *external)
{
    memset(g, 0, sizeof(*g));
    if (n_met <= 0 || n_rxn <= 0 || !row_ptr || !reversible || !external) return OR_EINVAL;
    if (row_ptr[0] != 0) return OR_EINVAL;
    for (int m = 0; m < n_met; ++m) {
        if (row_ptr[m + 1] < row_ptr[m]) return OR_EINVAL;
        for (int p = row_ptr[m]; p < row_ptr[m + 1]; ++p) {
            if (col_idx[p] < 0 || col_idx[p] >= n_rxn) return OR_EINVAL;
            if (coef[p] == 0 || coef[p] == INT32_MIN) return OR_EINVAL;
            for (int q = row_ptr[m]; q < p; ++q)
                if (col_idx[q] == col_idx[p]) return OR_EINVAL;
        }
    }
    g->n_met = n_met;
    g->n_rxn = n_rxn;
    int *first_col = (int *)malloc(sizeof(int) * (size_t)n_rxn);
    g->int_row = (int *)malloc(sizeof(int) * (size_t)n_met);
    if (!first_col || !g->int_row) { free(first_col); return OR_ENOMEM; }
    int N = 0;
    for (int j = 0; j < n_rxn; ++j) {
        first_col[j] = N;
        N += reversible[j] ? 2 : 1;
    }
    int M = 0;
    for (int m = 0; m < n_met; ++m) g->int_row[m] = external[m] ? -1 : M++;
    g->M = M;
    g->N = N;
    g->W = (N + 63) / 64;
    g->twin = (int *)malloc(sizeof(int) * (size_t)N);
    g->col_rxn = (int *)malloc(sizeof(int) * (size_t)N);
    g->col_dir = (int *)malloc(sizeof(int) * (size_t)N);
    g->S = (int64_t *)calloc((size_t)(M > 0 ? M : 1) * (size_t)N, sizeof(int64_t));
    g->deg_out = (int *)calloc((size_t)(M > 0 ? M : 1), sizeof(int));
    g->deg_in = (int *)calloc((size_t)(M > 0 ? M : 1), sizeof(int));
    if (!g->twin || !g->col_rxn || !g->col_dir || !g->S || !g->deg_out || !g->deg_in) {
        free(first_col);
        return OR_ENOMEM;
    }
    for (int j = 0; j < n_rxn; ++j) {
        int f = first_col[j];
        g->col_rxn[f] = j;
        g->col_dir[f] = 1;
        g->twin[f] = -1;
        if (reversible[j]) {
            g->col_rxn[f + 1] = j;
            g->col_dir[f + 1] = -1;
            g->twin[f] = f + 1;
            g->twin[f + 1] = f;
        }
    }
    for (int m = 0; m < n_met; ++m) {
        int r = g->int_row[m];
        if (r < 0) continue;
        for (int p = row_ptr[m]; p < row_ptr[m + 1]; ++p) {
            int j = col_idx[p];
            int f = first_col[j];
            g->S[(size_t)r * N + f] = coef[p];
            if (reversible[j]) g->S[(size_t)r * N + f + 1] = -(int64_t)coef[p];
        }
    }
    for (int r = 0; r < M; ++r)
        for (int k = 0; k < N; ++k) {
            int64_t s = g->S[(size_t)r * N + k];
            if (s < 0) g->deg_out[r]++;
            if (s > 0) g->deg_in[r]++;
        }
    free(first_col);
    return OR_OK;
}

/* S[t][col] over the full matrix (target row may be external). */
static int64_t full_coef(int t, int col, const or_net *g, const int32_t *row_ptr, const int32_t *col_idx,
                         const int32_t *coef)
{
    int j = g->col_rxn[col];
    for (int p = row_ptr[t]; p < row_ptr[t + 1]; ++p)
        if (col_idx[p] == j) return g->col_dir[col] * (int64_t)coef[p];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* dynamic arrays of fixed-size records                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint8_t *data;
    size_t n, cap, stride;
} vec;

static int vec_push(vec *v, const void *rec)
{
    if (v->n == v->cap) {
        size_t nc = v->cap ? v->cap * 2 : 256;
        uint8_t *p = (uint8_t *)realloc(v->data, nc * v->stride);
        if (!p) return -1;
        v->data = p;
        v->cap = nc;
    }
    memcpy(v->data + v->n * v->stride, rec, v->stride);
    v->n++;
    return 0;
}

static void *vec_at(const vec *v, size_t i) { return v->data + i * v->stride; }

/* state record: [U: W u64][EF: M i32][sec: i32]; key = U and EF */
static _Thread_local size_t g_keylen;

static int cmp_state(const void *a, const void *b) { return memcmp(a, b, g_keylen); }

/* set of supports (open addressing on W words) */
typedef struct {
    uint64_t *keys; /* cap * W */
    uint8_t *used;
    size_t cap, n;
    int W;
} supp_set;

static uint64_t supp_hash(const uint64_t *u, int W)
{
    uint64_t h = 0x9e3779b97f4a7c15ull;
    for (int w = 0; w < W; ++w) {
        h ^= u[w] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        h *= 0xff51afd7ed558ccdull;
    }
    return h ^ (h >> 33);
}

static int supp_set_grow(supp_set *s);

/* returns 1 if inserted (new), 0 if present, -1 on memory error */
static int supp_set_insert(supp_set *s, const uint64_t *u)
{
    if ((s->n + 1) * 2 > s->cap)
        if (supp_set_grow(s)) return -1;
    size_t pos = supp_hash(u, s->W) & (s->cap - 1);
    for (;;) {
        if (!s->used[pos]) {
            s->used[pos] = 1;
            memcpy(s->keys + pos * s->W, u, sizeof(uint64_t) * (size_t)s->W);
            s->n++;
            return 1;
        }
        if (memcmp(s->keys + pos * s->W, u, sizeof(uint64_t) * (size_t)s->W) == 0) return 0;
        pos = (pos + 1) & (s->cap - 1);
    }
}

static int supp_set_grow(supp_set *s)
{
    size_t nc = s->cap ? s->cap * 2 : 1024;
    supp_set t = {(uint64_t *)malloc(sizeof(uint64_t) * nc * (size_t)s->W), (uint8_t *)calloc(nc, 1), nc, 0,
                  s->W};
    if (!t.keys || !t.used) {
        free(t.keys);
        free(t.used);
        return -1;
    }
    for (size_t i = 0; i < s->cap; ++i)
        if (s->used[i]) supp_set_insert(&t, s->keys + i * s->W);
    free(s->keys);
    free(s->used);
    *s = t;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Arbiter: nullity of S_int[:, U] over Q equals 1                            */
/* ------------------------------------------------------------------------ */

static int is_elementary(const or_net *g, const uint64_t *U, int *out)
{
    int N = g->N, M = g->M;
    int n = 0;
    int *cols = (int *)malloc(sizeof(int) * (size_t)N);
    int *rows = (int *)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
    if (!cols || !rows) {
        free(cols);
        free(rows);
        return OR_ENOMEM;
    }
    for (int k = 0; k < N; ++k)
        if (bit_test(U, k)) cols[n++] = k;
    int r = 0;
    for (int i = 0; i < M; ++i) {
        int touched = 0;
        for (int j = 0; j < n; ++j)
            if (g->S[(size_t)i * N + cols[j]] != 0) { touched = 1; break; }
        if (touched) rows[r++] = i;
    }
    int rank = 0, rc = OR_OK;
    if (r > 0) {
        int64_t *A = (int64_t *)malloc(sizeof(int64_t) * (size_t)r * (size_t)n);
        if (!A) {
            free(cols);
            free(rows);
            return OR_ENOMEM;
        }
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = g->S[(size_t)rows[i] * N + cols[j]];
        rc = oracle_rank(r, n, A, 0, &rank);
        free(A);
    }
    free(cols);
    free(rows);
    if (rc != OR_OK) return rc;
    *out = (n - rank) == 1;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* output order: (|U|, ascending column list)                                 */
/* ------------------------------------------------------------------------ */

static _Thread_local int g_W;

static int cmp_support(const void *pa, const void *pb)
{
    const uint64_t *a = (const uint64_t *)pa, *b = (const uint64_t *)pb;
    int ca = popcount_words(a, g_W), cb = popcount_words(b, g_W);
    if (ca != cb) return ca < cb ? -1 : 1;
    /* equal sizes: compare the ascending column lists element by element */
    int ia = 0, ib = 0;
    int W = g_W;
    for (;;) {
        while (ia < W * 64 && !bit_test(a, ia)) ++ia;
        while (ib < W * 64 && !bit_test(b, ib)) ++ib;
        if (ia >= W * 64 || ib >= W * 64) return 0;
        if (ia != ib) return ia < ib ? -1 : 1;
        ++ia;
        ++ib;
    }
}

/* ------------------------------------------------------------------------ */
/* the traversal                                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    const or_net *g;
    const or_limits *lim;
    or_counters *ctr;
    supp_set seen;     /* balanced supports already judged */
    vec results;       /* records: [U: W u64][level: i64] */
} or_run;

/* judge a balanced support found at `level` */
static int judge(or_run *R, const uint64_t *U, int64_t level)
{
    int ins = supp_set_insert(&R->seen, U);
    if (ins < 0) return OR_ENOMEM;
    if (ins == 0) return OR_OK;
    R->ctr->candidates++;
    int efm = 0;
    int rc = is_elementary(R->g, U, &efm);
    if (rc != OR_OK) return rc;
    if (efm) {
        uint64_t rec[65];
        int W = R->g->W;
        memcpy(rec, U, sizeof(uint64_t) * (size_t)W);
        rec[W] = (uint64_t)level;
        if (vec_push(&R->results, rec)) return OR_ENOMEM;
        R->ctr->results++;
    }
    return OR_OK;
}

/* superset rule: the step that adds column k completes the support of a
 * result accepted before `level` (k in E and E contained in U + {k}) */
static int completes_result(const or_run *R, const uint64_t *U, int k, int64_t level)
{
    int W = R->g->W;
    for (size_t r = 0; r < R->results.n; ++r) {
        const uint64_t *E = (const uint64_t *)vec_at(&R->results, r);
        if ((int64_t)E[W] >= level) continue;
        if (!bit_test(E, k)) continue;
        int sub = 1;
        for (int w = 0; w < W; ++w)
            if (E[w] & ~U[w]) { sub = 0; break; }
        if (sub) return 1;
    }
    return 0;
}

/* EF / gcd(EF); returns 0 when every entry fits int32, 1 on overflow.
 * *zero is set when EF == 0 (balanced). */
static int normalise(const int64_t *ef, int M, int32_t *out, int *zero)
{
    uint64_t g = 0;
    for (int i = 0; i < M; ++i) g = gcd_u64(g, abs_i64(ef[i]));
    *zero = (g == 0);
    if (g == 0) {
        for (int i = 0; i < M; ++i) out[i] = 0;
        return 0;
    }
    int ovf = 0;
    for (int i = 0; i < M; ++i) {
        int64_t v = ef[i] / (int64_t)g;
        if (v > INT32_MAX || v < -(int64_t)INT32_MAX) ovf = 1;
        out[i] = (int32_t)v;
    }
    return ovf;
}

/* (EF, v) / gcd of all their entries (the subtractive variant's state ray);
 * returns 1 when some entry leaves the int32 range.  *zero: EF == 0. */
static int normalise2(const int64_t *ef, int M, const int64_t *v, int N, int32_t *ef_out, int32_t *v_out, int *zero)
{
    uint64_t g = 0;
    int nz = 0;
    for (int i = 0; i < M; ++i) {
        g = gcd_u64(g, abs_i64(ef[i]));
        nz |= ef[i] != 0;
    }
    for (int k = 0; k < N; ++k) g = gcd_u64(g, abs_i64(v[k]));
    *zero = !nz;
    if (g == 0) g = 1;
    int ovf = 0;
    for (int i = 0; i < M; ++i) {
        int64_t x = ef[i] / (int64_t)g;
        if (x > INT32_MAX || x < -(int64_t)INT32_MAX) ovf = 1;
        ef_out[i] = (int32_t)x;
    }
    for (int k = 0; k < N; ++k) {
        int64_t x = v[k] / (int64_t)g;
        if (x > INT32_MAX || x < -(int64_t)INT32_MAX) ovf = 1;
        v_out[k] = (int32_t)x;
    }
    return ovf;
}

/* Sort the child list and keep one record per key (the smallest sec). */
static void compact_children(vec *C, size_t key, size_t stride)
{
    g_keylen = key;
    qsort(C->data, C->n, stride, cmp_state);
    size_t u = 0;
    for (size_t i = 0; i < C->n; ++i) {
        uint8_t *ci = (uint8_t *)vec_at(C, i);
        if (u > 0) {
            uint8_t *cu = (uint8_t *)vec_at(C, u - 1);
            if (memcmp(cu, ci, key) == 0) {
                int32_t *su = (int32_t *)(cu + key), *si = (int32_t *)(ci + key);
                if (*si < *su) *su = *si;
                continue;
            }
        }
        if (u != i) memcpy(vec_at(C, u), ci, stride);
        ++u;
    }
    C->n = u;
}

/* Store a surviving child of a level.  With a frontier budget the list is
 * compacted (deduplicated) whenever it reaches 1.5 budgets; once it holds
 * more distinct states than the budget the level is truncated whatever
 * follows, so later children are no longer stored (*over; they are still
 * counted and judged by the caller).  This bounds the host memory of a
 * truncating level and changes no result or counter. */
static int push_child(vec *C, const uint8_t *rec, size_t key, size_t stride, const or_limits *lim, int *over)
{
    if (*over) return 0;
    if (lim->max_frontier > 0 && (int64_t)C->n >= lim->max_frontier + lim->max_frontier / 2 + 16) {
        compact_children(C, key, stride);
        if ((int64_t)C->n > lim->max_frontier) {
            *over = 1;
            return 0;
        }
    }
    return vec_push(C, rec);
}

/* The traversal from the seeds of a target (seedset == NULL), or from the
 * one state of a seed set R_in (Prop. 1): U = R_in with flux 1 on each of
 * its columns, EF = sum of their S_int columns / gcd, no secondary step,
 * at level |R_in| - 1 (a state's level is |U| - 1 + sec throughout). */
static int enumerate_impl(int32_t n_met, int32_t n_rxn, const int32_t *row_ptr, const int32_t *col_idx,
                          const int32_t *coef, const uint8_t *reversible, const uint8_t *external, int32_t target,
                          const int32_t *seedset, int32_t n_seedset, const or_limits *lim, uint64_t **out_supports,
                          int64_t *out_n, int32_t *out_W, or_counters *ctr)
{
    or_net g;
    int rc = net_build(&g, n_met, n_rxn, row_ptr, col_idx, coef, reversible, external);
    *out_supports = NULL;
    *out_n = 0;
    memset(ctr, 0, sizeof(*ctr));
    if (rc != OR_OK) {
        net_free(&g);
        return rc;
    }
    if (target < -1 || target >= n_met || lim->max_len < 1 || lim->max_len > 64 || lim->max_secondary < 0 ||
        g.W > 64) {
        net_free(&g);
        return OR_EINVAL;
    }
    if (seedset) {
        /* distinct columns, no twin pair, at most max_len of them */
        if (n_seedset < 1 || n_seedset > lim->max_len) {
            net_free(&g);
            return OR_EINVAL;
        }
        for (int a = 0; a < n_seedset; ++a) {
            if (seedset[a] < 0 || seedset[a] >= g.N) {
                net_free(&g);
                return OR_EINVAL;
            }
            for (int b = 0; b < a; ++b)
                if (seedset[b] == seedset[a] || g.twin[seedset[a]] == seedset[b]) {
                    net_free(&g);
                    return OR_EINVAL;
                }
        }
    }
    *out_W = g.W;
    const int M = g.M, N = g.N, W = g.W;
    const int sub = (lim->flags & OR_SUBTRACTIVE) != 0;
    const int NV = sub ? N : 0; /* flux entries kept per state */
    const int64_t level0 = seedset ? n_seedset - 1 : 0;
    /* record: U (W words), EF (M), v (NV), then sec; the key is all but sec */
    const size_t off_v = sizeof(uint64_t) * (size_t)W + sizeof(int32_t) * (size_t)M;
    const size_t key = off_v + sizeof(int32_t) * (size_t)NV;
    const size_t stride = key + sizeof(int32_t);
    or_run R;
    memset(&R, 0, sizeof(R));
    R.g = &g;
    R.lim = lim;
    R.ctr = ctr;
    R.seen.W = W;
    R.results.stride = sizeof(uint64_t) * (size_t)(W + 1);
    vec F = {NULL, 0, 0, stride}, C = {NULL, 0, 0, stride};
    uint8_t *rec = (uint8_t *)calloc(1, stride);
    int64_t *ef = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1));
    int32_t *efn = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    int64_t *vv = (int64_t *)calloc((size_t)(NV > 0 ? NV : 1), sizeof(int64_t));
    if (!rec || !ef || !efn || !vv) { rc = OR_ENOMEM; goto done; }

    /* level 0: seeds (INIT) -- or the one state of the seed set */
    for (int j = 0; j < (seedset ? 1 : N); ++j) {
        uint64_t *U = (uint64_t *)rec;
        memset(U, 0, sizeof(uint64_t) * (size_t)W);
        for (int k = 0; k < NV; ++k) vv[k] = 0;
        if (seedset) {
            for (int i = 0; i < M; ++i) ef[i] = 0;
            for (int a = 0; a < n_seedset; ++a) {
                const int k = seedset[a];
                for (int i = 0; i < M; ++i) ef[i] += g.S[(size_t)i * N + k]; /* Eq. 2, flux 1 on each */
                U[k >> 6] |= 1ull << (k & 63);
                if (sub) vv[k] = 1;
            }
        } else {
            if (target >= 0 && full_coef(target, j, &g, row_ptr, col_idx, coef) <= 0) continue;
            for (int i = 0; i < M; ++i) ef[i] = g.S[(size_t)i * N + j]; /* Eq. 2 with flux 1 on j */
            U[j >> 6] |= 1ull << (j & 63);
            if (sub) vv[j] = 1;
        }
        ctr->seeds++;
        int zero = 0;
        const int bad = sub ? normalise2(ef, M, vv, NV, (int32_t *)(rec + sizeof(uint64_t) * W),
                                         (int32_t *)(rec + off_v), &zero)
                            : normalise(ef, M, (int32_t *)(rec + sizeof(uint64_t) * W), &zero);
        if (bad) {
            ctr->overflow++;
            continue;
        }
        *(int32_t *)(rec + key) = 0;
        if (zero) {
            ctr->balanced++;
            if ((rc = judge(&R, U, level0)) != OR_OK) goto done;
        } else if (vec_push(&F, rec)) {
            rc = OR_ENOMEM;
            goto done;
        }
    }
    g_keylen = key;
    qsort(F.data, F.n, stride, cmp_state);
    ctr->levels = 1;
    if (lim->max_frontier > 0 && (int64_t)F.n > lim->max_frontier) {
        ctr->status |= OR_TRUNCATED;
        goto finish;
    }
    ctr->frontier += (int64_t)F.n;
    if ((int64_t)F.n > ctr->frontier_max) ctr->frontier_max = (int64_t)F.n;
    if (lim->max_results > 0 && ctr->results >= lim->max_results) {
        ctr->status |= OR_CAPPED;
        goto finish;
    }

    for (int64_t level = level0 + 1; F.n > 0; ++level) {
        C.n = 0;
        int over = 0; /* the level already holds more distinct states than the budget */
        for (size_t s = 0; s < F.n; ++s) {
            const uint8_t *st = (const uint8_t *)vec_at(&F, s);
            const uint64_t *U = (const uint64_t *)st;
            const int32_t *EF = (const int32_t *)(st + sizeof(uint64_t) * W);
            const int32_t *V = (const int32_t *)(st + off_v); /* flux vector (subtractive variant) */
            const int32_t sec = *(const int32_t *)(st + key);
            const int pc = popcount_words(U, W);
            /* acting metabolite: fewest reactions able to balance it, then index */
            int piv = -1, best = 0;
            for (int i = 0; i < M; ++i) {
                if (EF[i] == 0) continue;
                int d = EF[i] > 0 ? g.deg_out[i] : g.deg_in[i];
                if (piv < 0 || d < best) { piv = i; best = d; }
            }
            if (piv < 0) continue; /* cannot happen: frontier states are unbalanced */
            const int64_t ef_i = EF[piv];
            for (int k = 0; k < N; ++k) {
                const int64_t s_ik = g.S[(size_t)piv * N + k];
                /* forward flow (EF_i > 0): outputs of i; backward: inputs */
                if (!(ef_i > 0 ? s_ik < 0 : s_ik > 0)) continue;
                if (g.twin[k] >= 0 && bit_test(U, g.twin[k])) continue;
                const int in_u = bit_test(U, k);
                if (!in_u && pc + 1 > lim->max_len) continue;
                if (in_u && sec + 1 > lim->max_secondary) continue;
                ctr->expansions++;
                /* Eq. 3 in integers.  No int64 overflow: |EF[i]| <= 2^31 - 1
                 * (normalise() drops wider rows), a <= |S_ik| <= 2^31 - 1 and
                 * c <= |EF_i| (net_build() refuses INT32_MIN), so each product is
                 * below 2^62 and the sum below 2^63. */
                const uint64_t g0 = gcd_u64(abs_i64(ef_i), abs_i64(s_ik));
                const int64_t a = (int64_t)(abs_i64(s_ik) / g0);
                const int64_t c = (int64_t)(abs_i64(ef_i) / g0);
                for (int i = 0; i < M; ++i) ef[i] = a * (int64_t)EF[i] + c * g.S[(size_t)i * N + k];
                for (int x = 0; x < NV; ++x) vv[x] = a * (int64_t)V[x];
                if (sub) vv[k] += c;
                uint64_t *U2 = (uint64_t *)rec;
                memcpy(U2, U, sizeof(uint64_t) * (size_t)W);
                U2[k >> 6] |= 1ull << (k & 63);
                int zero = 0;
                const int bad = sub ? normalise2(ef, M, vv, NV, (int32_t *)(rec + sizeof(uint64_t) * W),
                                                 (int32_t *)(rec + off_v), &zero)
                                    : normalise(ef, M, (int32_t *)(rec + sizeof(uint64_t) * W), &zero);
                if (bad) {
                    ctr->overflow++;
                    continue;
                }
                *(int32_t *)(rec + key) = sec + in_u;
                if (zero) {
                    ctr->balanced++;
                    if ((rc = judge(&R, U2, level)) != OR_OK) goto done;
                    continue;
                }
                if (!in_u && !(lim->flags & OR_NO_PRUNE) && completes_result(&R, U2, k, level)) {
                    ctr->pruned++;
                    continue;
                }
                if (push_child(&C, rec, key, stride, lim, &over)) {
                    rc = OR_ENOMEM;
                    goto done;
                }
            }
            /* Eq. 5: take flux away from a reaction k in U that moves the
             * acting metabolite the same way as its imbalance */
            for (int k = 0; k < N && sub; ++k) {
                const int64_t s_ik = g.S[(size_t)piv * N + k];
                if (!(ef_i > 0 ? s_ik > 0 : s_ik < 0)) continue;
                if (!bit_test(U, k)) continue;
                if (sec + 1 > lim->max_secondary) continue;
                ctr->expansions++;
                const uint64_t g0 = gcd_u64(abs_i64(ef_i), abs_i64(s_ik));
                const int64_t a = (int64_t)(abs_i64(s_ik) / g0);
                const int64_t c = (int64_t)(abs_i64(ef_i) / g0);
                for (int i = 0; i < M; ++i) ef[i] = a * (int64_t)EF[i] - c * g.S[(size_t)i * N + k];
                for (int x = 0; x < NV; ++x) vv[x] = a * (int64_t)V[x];
                vv[k] -= c;
                if (vv[k] <= 0) { /* Prop. 3: no flux left on k (or less than none) */
                    ctr->zero_flux++;
                    continue;
                }
                uint64_t *U2 = (uint64_t *)rec;
                memcpy(U2, U, sizeof(uint64_t) * (size_t)W);
                int zero = 0;
                if (normalise2(ef, M, vv, NV, (int32_t *)(rec + sizeof(uint64_t) * W), (int32_t *)(rec + off_v),
                               &zero)) {
                    ctr->overflow++;
                    continue;
                }
                *(int32_t *)(rec + key) = sec + 1;
                if (zero) {
                    ctr->balanced++;
                    if ((rc = judge(&R, U2, level)) != OR_OK) goto done;
                    continue;
                }
                if (push_child(&C, rec, key, stride, lim, &over)) {
                    rc = OR_ENOMEM;
                    goto done;
                }
            }
        }
        /* F_level = distinct (U, EF) of the surviving children (with v in
         * the subtractive variant) */
        compact_children(&C, key, stride);
        vec t = F;
        F = C;
        C = t;
        ctr->levels = level - level0 + 1;
        if (over || (lim->max_frontier > 0 && (int64_t)F.n > lim->max_frontier)) {
            ctr->status |= OR_TRUNCATED;
            break;
        }
        ctr->frontier += (int64_t)F.n;
        if ((int64_t)F.n > ctr->frontier_max) ctr->frontier_max = (int64_t)F.n;
        if (lim->max_results > 0 && ctr->results >= lim->max_results) {
            ctr->status |= OR_CAPPED;
            break;
        }
    }

finish:
    if (ctr->overflow) ctr->status |= OR_OVERFLOW_DROPPED;
    {
        size_t n = R.results.n;
        uint64_t *out = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W * (n > 0 ? n : 1));
        if (!out) { rc = OR_ENOMEM; goto done; }
        for (size_t r = 0; r < n; ++r)
            memcpy(out + r * W, vec_at(&R.results, r), sizeof(uint64_t) * (size_t)W);
        g_W = W;
        qsort(out, n, sizeof(uint64_t) * (size_t)W, cmp_support);
        if (lim->max_results > 0 && (int64_t)n > lim->max_results) n = (size_t)lim->max_results;
        *out_supports = out;
        *out_n = (int64_t)n;
    }
    rc = OR_OK;
done:
    free(rec);
    free(ef);
    free(efn);
    free(vv);
    free(F.data);
    free(C.data);
    free(R.results.data);
    free(R.seen.keys);
    free(R.seen.used);
    net_free(&g);
    return rc;
}

int oracle_enumerate(int32_t n_met, int32_t n_rxn, const int32_t *row_ptr, const int32_t *col_idx,
                     const int32_t *coef, const uint8_t *reversible, const uint8_t *external, int32_t target,
                     const or_limits *lim, uint64_t **out_supports, int64_t *out_n, int32_t *out_W,
                     or_counters *ctr)
{
    return enumerate_impl(n_met, n_rxn, row_ptr, col_idx, coef, reversible, external, target, NULL, 0, lim,
                          out_supports, out_n, out_W, ctr);
}

int oracle_enumerate_from(int32_t n_met, int32_t n_rxn, const int32_t *row_ptr, const int32_t *col_idx,
                          const int32_t *coef, const uint8_t *reversible, const uint8_t *external,
                          const int32_t *seedset, int32_t n_seedset, const or_limits *lim, uint64_t **out_supports,
                          int64_t *out_n, int32_t *out_W, or_counters *ctr)
{
    if (!seedset) return OR_EINVAL;
    return enumerate_impl(n_met, n_rxn, row_ptr, col_idx, coef, reversible, external, -1, seedset, n_seedset, lim,
                          out_supports, out_n, out_W, ctr);
}

/* ------------------------------------------------------------------------ */
/* Monte-Carlo mode: the paper's own random walks                            */
/* ------------------------------------------------------------------------ */

/* The random number of counter c under key `seed`: the first output of the
 * SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014) started from
 * state seed + c * 0x9E3779B97F4A7C15. */
static uint64_t splitmix_at(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix_at(uint64_t seed, uint64_t c) { return splitmix_at(seed, c); }

/*
 * Walk w of n_walks (INIT then METAx of Alg. 3 with its random choices, in
 * the exact integer form of the exhaustive traversal):
 *   counter base c0 = 128 w;
 *   seed column = the (r(c0) mod n)-th of the target's n seed columns in
 *   ascending order (every column for target -1), EF = S_int[:, j] / gcd;
 *   step s = 1, 2, ...: a balanced EF ends the walk (its support is judged
 *   once per run, like the traversal's); otherwise the acting metabolite is
 *   chosen as in the traversal, its valid branches (ascending columns, the
 *   traversal's twin and length / secondary rules) are counted, none ends
 *   the walk as a dead end, else branch number r(c0 + s) mod count is taken
 *   and the AND update applied (an entry outside int32 ends the walk as
 *   overflow).
 * Counters: seeds = walks started, expansions = AND updates, overflow and
 * balanced = walks ended so, pruned = walks ended at a dead end,
 * levels = the most steps of a walk; frontier counters stay 0.
 */
int oracle_sample(int32_t n_met, int32_t n_rxn, const int32_t *row_ptr, const int32_t *col_idx,
                  const int32_t *coef, const uint8_t *reversible, const uint8_t *external, int32_t target,
                  const or_limits *lim, uint64_t seed, int64_t n_walks, uint64_t **out_supports, int64_t *out_n,
                  int32_t *out_W, or_counters *ctr)
{
    or_net g;
    int rc = net_build(&g, n_met, n_rxn, row_ptr, col_idx, coef, reversible, external);
    *out_supports = NULL;
    *out_n = 0;
    memset(ctr, 0, sizeof(*ctr));
    if (rc != OR_OK) {
        net_free(&g);
        return rc;
    }
    if (target < -1 || target >= n_met || lim->max_len < 1 || lim->max_len > 64 || lim->max_secondary < 0 ||
        lim->max_secondary > 63 || n_walks < 0 || g.W > 64) {
        net_free(&g);
        return OR_EINVAL;
    }
    *out_W = g.W;
    const int M = g.M, N = g.N, W = g.W;
    or_run R;
    memset(&R, 0, sizeof(R));
    R.g = &g;
    R.lim = lim;
    R.ctr = ctr;
    R.seen.W = W;
    R.results.stride = sizeof(uint64_t) * (size_t)(W + 1);
    int *seeds = (int *)malloc(sizeof(int) * (size_t)N);
    int *valid = (int *)malloc(sizeof(int) * (size_t)N);
    int64_t *ef = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1));
    int32_t *EF = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    uint64_t U[64];
    if (!seeds || !valid || !ef || !EF) { rc = OR_ENOMEM; goto done; }
    int n_seeds = 0;
    for (int j = 0; j < N; ++j)
        if (target < 0 || full_coef(target, j, &g, row_ptr, col_idx, coef) > 0) seeds[n_seeds++] = j;
    for (int64_t w = 0; w < n_walks && n_seeds > 0; ++w) {
        const uint64_t c0 = (uint64_t)w * 128u;
        const int j = seeds[splitmix_at(seed, c0) % (uint64_t)n_seeds];
        ctr->seeds++;
        memset(U, 0, sizeof(U));
        U[j >> 6] |= 1ull << (j & 63);
        for (int i = 0; i < M; ++i) ef[i] = g.S[(size_t)i * N + j];
        int zero = 0, pc = 1, sec = 0;
        int64_t steps = 0;
        if (normalise(ef, M, EF, &zero)) {
            ctr->overflow++;
            continue;
        }
        for (int s = 1;; ++s) {
            if (zero) {
                ctr->balanced++;
                if ((rc = judge(&R, U, 0)) != OR_OK) goto done;
                break;
            }
            int piv = -1, best = 0;
            for (int i = 0; i < M; ++i) {
                if (EF[i] == 0) continue;
                int d = EF[i] > 0 ? g.deg_out[i] : g.deg_in[i];
                if (piv < 0 || d < best) { piv = i; best = d; }
            }
            const int64_t ef_i = EF[piv];
            int n_valid = 0;
            for (int k = 0; k < N; ++k) {
                const int64_t s_ik = g.S[(size_t)piv * N + k];
                if (!(ef_i > 0 ? s_ik < 0 : s_ik > 0)) continue;
                if (g.twin[k] >= 0 && bit_test(U, g.twin[k])) continue;
                const int in_u = bit_test(U, k);
                if (!in_u && pc + 1 > lim->max_len) continue;
                if (in_u && sec + 1 > lim->max_secondary) continue;
                valid[n_valid++] = k;
            }
            if (n_valid == 0) {
                ctr->pruned++;
                break;
            }
            const int k = valid[splitmix_at(seed, c0 + (uint64_t)s) % (uint64_t)n_valid];
            const int64_t s_ik = g.S[(size_t)piv * N + k];
            ctr->expansions++;
            ++steps;
            const uint64_t g0 = gcd_u64(abs_i64(ef_i), abs_i64(s_ik));
            const int64_t a = (int64_t)(abs_i64(s_ik) / g0);
            const int64_t c = (int64_t)(abs_i64(ef_i) / g0);
            for (int i = 0; i < M; ++i) ef[i] = a * (int64_t)EF[i] + c * g.S[(size_t)i * N + k];
            if (bit_test(U, k)) {
                ++sec;
            } else {
                U[k >> 6] |= 1ull << (k & 63);
                ++pc;
            }
            if (normalise(ef, M, EF, &zero)) {
                ctr->overflow++;
                break;
            }
        }
        if (steps > ctr->levels) ctr->levels = steps;
    }
    if (ctr->overflow) ctr->status |= OR_OVERFLOW_DROPPED;
    {
        size_t n = R.results.n;
        uint64_t *out = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W * (n > 0 ? n : 1));
        if (!out) { rc = OR_ENOMEM; goto done; }
        for (size_t r = 0; r < n; ++r)
            memcpy(out + r * W, vec_at(&R.results, r), sizeof(uint64_t) * (size_t)W);
        g_W = W;
        qsort(out, n, sizeof(uint64_t) * (size_t)W, cmp_support);
        *out_supports = out;
        *out_n = (int64_t)n;
    }
    rc = OR_OK;
done:
    free(seeds);
    free(valid);
    free(ef);
    free(EF);
    free(R.results.data);
    free(R.seen.keys);
    free(R.seen.used);
    net_free(&g);
    return rc;
}

/* column -> (original reaction, direction), as used for supports */
int oracle_column_map(int32_t n_rxn, const uint8_t *reversible, int32_t *col_rxn, int32_t *col_dir)
{
    int N = 0;
    for (int j = 0; j < n_rxn; ++j) {
        col_rxn[N] = j;
        col_dir[N++] = 1;
        if (reversible[j]) {
            col_rxn[N] = j;
            col_dir[N++] = -1;
        }
    }
    return N;
}

void oracle_free(void *p) { free(p); }
