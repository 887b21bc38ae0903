/*
 * cg_oracle.c -- FP64 CPU oracle for the CountGauss transform T.X = G.(S.X).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code with the CUDA library: its random-number generator, its
 * hash, its Box-Muller step and its scatter are written here, separately.
 *
 * What the paper fixes (Kapralov, Potluru, Woodruff, "How to Fake Multiply by a
 * Gaussian Matrix"):
 *   - S is a B x n CountSketch: every column i of S holds exactly one nonzero, at a
 *     uniformly random row h(i), with value sigma(i) = +1 or -1 with probability 1/2,
 *     all choices independent (Section 1.1 "Our Results"; Section 7 first paragraph;
 *     the proof of Lemma 5 names the position h(k) and value sigma(k)).
 *   - G is an m x B matrix of i.i.d. unit-variance Gaussians, G~ an m x n one
 *     (Section 2, Theorem 1).  No 1/sqrt(m) scaling is applied.
 *   - T = G.S and the product is computed as T.X = G.(S.X) (Section 1.1; Algorithm 1
 *     steps 1-2).  The plain product it replaces is G~.X (Abstract; Section 4).
 *   - The SVM application projects a samples x features matrix X to X.R with
 *     R = T^T (Section 9; Table 1 times this projection).
 *
 * What the paper leaves open and this project fixes (the "stream layout"):
 *   - Random words come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 *     Random Numbers: As Easy as 1, 2, 3", SC'11): key = (lo32(seed), hi32(seed)),
 *     counter = (lo32(idx), hi32(idx), tag, 0).
 *   - tag 0, idx = floor(i / 4) for global row i: with w = word (i mod 4) of that
 *     call, h(i) = floor(w * B / 2^32) and sigma(i) = -1 if the lowest bit of w is set,
 *     else +1 (one call serves four consecutive rows).
 *   - uniform u(w) = (2 * (w >> 9) + 1) * 2^-24, an odd multiple of 2^-24 in (0,1).
 *   - an R x C Gaussian matrix with tag t: entry (r, c) is lane (r mod 4) of the four
 *     Box-Muller normals from the Philox call at idx = c * ceil(R/4) + floor(r/4):
 *       z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1),
 *       z2 = sqrt(-2 ln u2) cos(2 pi u3), z3 = sqrt(-2 ln u2) sin(2 pi u3).
 *     G uses tag 1 (R = m, C = B), G~ uses tag 2 (R = m, C = n, c = global row).
 *
 * Everything is computed in double precision in the plain order of the definitions.
 * Each routine is deliberately naive.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_HASH 0u
#define ORC_TAG_G 1u
#define ORC_TAG_GTILDE 2u

static const double ORC_TWO_PI = 6.283185307179586476925286766559;

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (SC'11).  Ten rounds of the 4x32 Philox S-box with the two round
 * multipliers, and the key bumped by the two Weyl constants between rounds.
 * ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The four words for (seed, idx, tag) under the project's stream layout (all randomness
 * is a function of a short seed, as Section 4 allows). */
static void orc_words(uint64_t seed, uint64_t idx, uint32_t tag, uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    ctr[0] = (uint32_t)(idx & 0xffffffffu);
    ctr[1] = (uint32_t)(idx >> 32);
    ctr[2] = tag;
    ctr[3] = 0u;
    orc_philox4x32_10(ctr, key, out);
}

/* Batch form for the tests: words for idx = idx0 .. idx0+count-1, out is count x 4. */
void orc_philox_words(uint64_t seed, uint32_t tag, uint64_t idx0, int64_t count, uint32_t *out)
{
    int64_t t;
    for (t = 0; t < count; ++t)
        orc_words(seed, idx0 + (uint64_t)t, tag, out + 4 * t);
}

/* ---------------------------------------------------------------------------
 * Column hash h and sign sigma of the CountSketch (Section 1.1; Section 7).
 * Row i takes word (i mod 4) of the tag-0 call at idx floor(i/4).  h(i) is uniform on
 * [0, B) (multiply-high of a uniform 32-bit word, bias at most B / 2^32); sigma(i) is
 * its lowest bit, which is independent of h(i) when B is a power of two (h then reads
 * only the top log2(B) bits) and otherwise tilts P(sigma = -1 | h) from 1/2 by at most
 * B / 2^32 (B < 2^31: each bucket is an interval of at least two words, whose odd
 * words are half of them up to one).  Different rows use different words, so all
 * choices are independent.
 * ------------------------------------------------------------------------- */
static void orc_hash_sign_one(uint64_t seed, int64_t B, int64_t i, int64_t *h, int *sigma)
{
    uint32_t w[4];
    uint32_t x;
    orc_words(seed, (uint64_t)i / 4u, ORC_TAG_HASH, w);
    x = w[(uint64_t)i % 4u];
    *h = (int64_t)(((uint64_t)x * (uint64_t)B) >> 32);
    *sigma = (x & 1u) ? -1 : 1;
}

void orc_hash_sign(uint64_t seed, int64_t B, int64_t row0, int64_t count, int64_t *h, int32_t *sigma)
{
    int64_t t;
    for (t = 0; t < count; ++t) {
        int s;
        orc_hash_sign_one(seed, B, row0 + t, &h[t], &s);
        sigma[t] = s;
    }
}

/* Uniform in (0,1) from a 32-bit word: odd multiples of 2^-24, exact in double. */
double orc_uniform24(uint32_t w)
{
    return (double)(2u * (w >> 9) + 1u) * (1.0 / 16777216.0);
}

/* Box-Muller (Box and Muller, 1958): the four unit-variance normals of one Philox
 * call, the N(0,1) entries Theorem 1 asks of G and G~. */
static void orc_box_muller4(const uint32_t w[4], double z[4])
{
    double u0 = orc_uniform24(w[0]), u1 = orc_uniform24(w[1]);
    double u2 = orc_uniform24(w[2]), u3 = orc_uniform24(w[3]);
    double rad01 = sqrt(-2.0 * log(u0));
    double rad23 = sqrt(-2.0 * log(u2));
    z[0] = rad01 * cos(ORC_TWO_PI * u1);
    z[1] = rad01 * sin(ORC_TWO_PI * u1);
    z[2] = rad23 * cos(ORC_TWO_PI * u3);
    z[3] = rad23 * sin(ORC_TWO_PI * u3);
}

void orc_box_muller_words(const uint32_t *w, int64_t count, double *z)
{
    int64_t t;
    for (t = 0; t < count; ++t)
        orc_box_muller4(w + 4 * t, z + 4 * t);
}

/* One entry (r, c) of the R x C Gaussian matrix with tag `tag` (G: Section 2,
 * Theorem 1; G~: Abstract). */
static double orc_gauss_entry(uint64_t seed, uint32_t tag, int64_t R, int64_t r, int64_t c)
{
    uint32_t w[4];
    double z[4];
    int64_t groups = (R + 3) / 4;
    orc_words(seed, (uint64_t)c * (uint64_t)groups + (uint64_t)(r / 4), tag, w);
    orc_box_muller4(w, z);
    return z[r % 4];
}

/* Column c of the R x C Gaussian matrix, all R entries (one Philox call per group
 * of four rows). */
static void orc_gauss_column(uint64_t seed, uint32_t tag, int64_t R, int64_t c, double *col)
{
    int64_t groups = (R + 3) / 4, g, r;
    for (g = 0; g < groups; ++g) {
        uint32_t w[4];
        double z[4];
        orc_words(seed, (uint64_t)c * (uint64_t)groups + (uint64_t)g, tag, w);
        orc_box_muller4(w, z);
        for (r = 4 * g; r < 4 * g + 4 && r < R; ++r)
            col[r] = z[r - 4 * g];
    }
}

/* Sub-block rows [r0,r1) x cols [c0,c1) of the R x C Gaussian matrix with tag `tag`,
 * row-major into out ((r1-r0) x (c1-c0)).  Entry by entry, straight from the layout. */
void orc_gaussian_block(uint64_t seed, uint32_t tag, int64_t R, int64_t r0, int64_t r1,
                        int64_t c0, int64_t c1, double *out)
{
    int64_t r, c, w = c1 - c0;
    for (r = r0; r < r1; ++r)
        for (c = c0; c < c1; ++c)
            out[(r - r0) * w + (c - c0)] = orc_gauss_entry(seed, tag, R, r, c);
}

/* ---------------------------------------------------------------------------
 * S.X for CSR X (Section 1.1: S.X costs O(nnz(X))).  X has n local rows whose
 * global indices are row_offset .. row_offset+n-1; row i contributes sigma(i) X[i,:]
 * to row h(i) of SX.  SX is B x d, row-major, overwritten.
 * ------------------------------------------------------------------------- */
void orc_sketch_csr(uint64_t seed, int64_t n, int64_t d, int64_t B, int64_t row_offset,
                    const int64_t *row_ptr, const int64_t *col_idx, const double *vals, double *SX)
{
    int64_t i, k;
    memset(SX, 0, (size_t)(B * d) * sizeof(double));
    for (i = 0; i < n; ++i) {
        int64_t h;
        int s;
        orc_hash_sign_one(seed, B, row_offset + i, &h, &s);
        for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            SX[h * d + col_idx[k]] += (double)s * vals[k];
    }
}

/* S.X for dense row-major X (n x d) (Section 1.1). */
void orc_sketch_dense(uint64_t seed, int64_t n, int64_t d, int64_t B, int64_t row_offset,
                      const double *X, double *SX)
{
    int64_t i, j;
    memset(SX, 0, (size_t)(B * d) * sizeof(double));
    for (i = 0; i < n; ++i) {
        int64_t h;
        int s;
        orc_hash_sign_one(seed, B, row_offset + i, &h, &s);
        for (j = 0; j < d; ++j)
            SX[h * d + j] += (double)s * X[i * d + j];
    }
}

/* The part of Y = G.SX (Section 2, Theorem 1; Algorithm 1 step 2) that columns
 * b0 <= b < b1 of G contribute: the sum over those b of the outer products
 * G[:,b] SX[b,:], each column of G generated once.  SX holds all B rows (B x d,
 * row-major); Y is m x d row-major, overwritten. */
void orc_contract_range(uint64_t seed, int64_t m, int64_t B, int64_t d, int64_t b0, int64_t b1,
                        const double *SX, double *Y)
{
    int64_t b, r, j;
    double *g = (double *)malloc((size_t)m * sizeof(double));
    memset(Y, 0, (size_t)(m * d) * sizeof(double));
    if (b0 < 0) b0 = 0;
    if (b1 > B) b1 = B;
    for (b = b0; b < b1; ++b) {
        orc_gauss_column(seed, ORC_TAG_G, m, b, g);
        for (r = 0; r < m; ++r)
            for (j = 0; j < d; ++j)
                Y[r * d + j] += g[r] * SX[b * d + j];
    }
    free(g);
}

/* Y = G.SX with G the m x B Gaussian of tag 1: all columns b of G, in order. */
void orc_contract(uint64_t seed, int64_t m, int64_t B, int64_t d, const double *SX, double *Y)
{
    orc_contract_range(seed, m, B, d, 0, B, SX, Y);
}

/* T.X = G.(S.X) for CSR X (Section 1.1; Algorithm 1 steps 1-2).  SX (B x d) is
 * returned too, for stage-wise checks. */
void orc_apply_csr(uint64_t seed, int64_t n, int64_t d, int64_t m, int64_t B, int64_t row_offset,
                   const int64_t *row_ptr, const int64_t *col_idx, const double *vals,
                   double *SX, double *Y)
{
    orc_sketch_csr(seed, n, d, B, row_offset, row_ptr, col_idx, vals, SX);
    orc_contract(seed, m, B, d, SX, Y);
}

/* T.X = G.(S.X) for dense X (Section 1.1; Algorithm 1 steps 1-2). */
void orc_apply_dense(uint64_t seed, int64_t n, int64_t d, int64_t m, int64_t B, int64_t row_offset,
                     const double *X, double *SX, double *Y)
{
    orc_sketch_dense(seed, n, d, B, row_offset, X, SX);
    orc_contract(seed, m, B, d, SX, Y);
}

/* ---------------------------------------------------------------------------
 * The random projection X.R of the SVM application (Section 9, the theorem on the
 * margin; Table 1's "Proj" column), with R = T^T.  Here the data matrix A has one row
 * per sample (d rows) and one column per feature (n columns), the orientation of
 * Section 9, and Z = A.T^T is d x m.  Written from the definition T = G.S: column c
 * of T is sigma(c) G[:, h(c)], so the nonzero A[r, c] adds A[r, c] sigma(c) G[:, h(c)]
 * to row r of Z.  Column c of A carries the global index col_offset + c (the index
 * T's column is drawn for).  Z is d x m row-major, overwritten.
 * ------------------------------------------------------------------------- */
void orc_apply_right_csr(uint64_t seed, int64_t n, int64_t d, int64_t m, int64_t B, int64_t col_offset,
                         const int64_t *row_ptr, const int64_t *col_idx, const double *vals, double *Z)
{
    int64_t r, k, q;
    double *g = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    (void)n;
    memset(Z, 0, (size_t)(d * m) * sizeof(double));
    for (r = 0; r < d; ++r) {
        for (k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
            int64_t h;
            int s;
            orc_hash_sign_one(seed, B, col_offset + col_idx[k], &h, &s);
            orc_gauss_column(seed, ORC_TAG_G, m, h, g);
            for (q = 0; q < m; ++q)
                Z[r * m + q] += vals[k] * (double)s * g[q];
        }
    }
    free(g);
}

/* ---------------------------------------------------------------------------
 * The plain product G~.X that the method replaces (Abstract; Section 4), G~ the
 * m x n_global Gaussian of tag 2 whose column index is the global row of X.
 * Only the output rows listed in rows[0..nsel) are formed (row r of the result
 * depends on row r of G~ alone); Ysel is nsel x d row-major, overwritten.
 * ------------------------------------------------------------------------- */
void orc_plain_csr(uint64_t seed, int64_t n, int64_t d, int64_t m, int64_t row_offset,
                   const int64_t *row_ptr, const int64_t *col_idx, const double *vals,
                   int64_t nsel, const int64_t *rows, double *Ysel)
{
    int64_t i, k, t, groups = (m + 3) / 4;
    memset(Ysel, 0, (size_t)(nsel * d) * sizeof(double));
    for (i = 0; i < n; ++i) {
        int64_t last_group = -1;
        double z[4];
        if (row_ptr[i] == row_ptr[i + 1])
            continue; /* column i of G~ meets only zeros of X */
        for (t = 0; t < nsel; ++t) {
            /* entry (rows[t], global row) of G~; consecutive selected rows of the same
             * group of four share one Philox call */
            int64_t grp = rows[t] / 4;
            double g;
            if (grp != last_group) {
                uint32_t w[4];
                orc_words(seed, (uint64_t)(row_offset + i) * (uint64_t)groups + (uint64_t)grp,
                          ORC_TAG_GTILDE, w);
                orc_box_muller4(w, z);
                last_group = grp;
            }
            g = z[rows[t] % 4];
            for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                Ysel[t * d + col_idx[k]] += g * vals[k];
        }
    }
}

/* Plain product G~.X for dense X, all m rows (Abstract; Section 4). */
void orc_plain_dense(uint64_t seed, int64_t n, int64_t d, int64_t m, int64_t row_offset,
                     const double *X, double *Y)
{
    int64_t i, r, j;
    double *g = (double *)malloc((size_t)m * sizeof(double));
    memset(Y, 0, (size_t)(m * d) * sizeof(double));
    for (i = 0; i < n; ++i) {
        orc_gauss_column(seed, ORC_TAG_GTILDE, m, row_offset + i, g);
        for (r = 0; r < m; ++r)
            for (j = 0; j < d; ++j)
                Y[r * d + j] += g[r] * X[i * d + j];
    }
    free(g);
}

/* ---------------------------------------------------------------------------
 * Adjoint.  T is linear (Section 1.1), so the gradient of <T.X, dY> with respect
 * to X is T^T dY = S^T (G^T dY).
 * W = G^T dY is B x d; dX[i,:] = sigma(i) W[h(i),:] for dense X, and for CSR X the
 * same expression read at the stored nonzeros only.
 * ------------------------------------------------------------------------- */
void orc_adjoint_w(uint64_t seed, int64_t m, int64_t B, int64_t d, const double *dY, double *W)
{
    int64_t b, r, j;
    double *g = (double *)malloc((size_t)m * sizeof(double));
    for (b = 0; b < B; ++b) {
        orc_gauss_column(seed, ORC_TAG_G, m, b, g);
        for (j = 0; j < d; ++j) {
            double acc = 0.0;
            for (r = 0; r < m; ++r)
                acc += g[r] * dY[r * d + j];
            W[b * d + j] = acc;
        }
    }
    free(g);
}

void orc_adjoint_dense(uint64_t seed, int64_t n, int64_t d, int64_t m, int64_t B, int64_t row_offset,
                       const double *dY, double *W, double *dX)
{
    int64_t i, j;
    orc_adjoint_w(seed, m, B, d, dY, W);
    for (i = 0; i < n; ++i) {
        int64_t h;
        int s;
        orc_hash_sign_one(seed, B, row_offset + i, &h, &s);
        for (j = 0; j < d; ++j)
            dX[i * d + j] = (double)s * W[h * d + j];
    }
}

void orc_adjoint_csr(uint64_t seed, int64_t n, int64_t d, int64_t m, int64_t B, int64_t row_offset,
                     const int64_t *row_ptr, const int64_t *col_idx, const double *dY,
                     double *W, double *dXvals)
{
    int64_t i, k;
    orc_adjoint_w(seed, m, B, d, dY, W);
    for (i = 0; i < n; ++i) {
        int64_t h;
        int s;
        orc_hash_sign_one(seed, B, row_offset + i, &h, &s);
        for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            dXvals[k] = (double)s * W[h * d + col_idx[k]];
    }
}

/* ---------------------------------------------------------------------------
 * Algorithm 1 step 3 (NMF anchors): for every row r of Z = T.X, the column index of
 * its maximum and of its minimum.  Ties go to the lowest column index.
 * ------------------------------------------------------------------------- */
void orc_row_argmax_argmin(int64_t m, int64_t d, const double *Z, int64_t *imax, int64_t *imin)
{
    int64_t r, j;
    for (r = 0; r < m; ++r) {
        int64_t bmax = 0, bmin = 0;
        for (j = 1; j < d; ++j) {
            if (Z[r * d + j] > Z[r * d + bmax]) bmax = j;
            if (Z[r * d + j] < Z[r * d + bmin]) bmin = j;
        }
        imax[r] = bmax;
        imin[r] = bmin;
    }
}
