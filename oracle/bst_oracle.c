/*
 * bst_oracle.c -- plain, slow, obviously correct CPU oracle for the block-sparse
 * multiply and the block-sparse tensor contraction of DBCSR (arXiv:1910.13555).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link, load
 * or call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or table with the CUDA library.
 *
 * Everything is FP64, plain loops, no BLAS, compiled with -ffp-contract=off so that
 * every multiply and add rounds separately in the order written here.
 *
 * What it follows:
 *   - Paper Sec. 2: a matrix is stored as blocks in blocked-CSR form; the local
 *     multiplication is made of pairwise products of small dense blocks,
 *     an (m x k) block of A times a (k x n) block of B, accumulated into C
 *     ("C = C + A x B").  Blocks of A are visited row-block by row-block and, for
 *     each, the matching blocks of B.
 *   - Paper Sec. 3.1: the S_C << S_A,S_B case multiplies the transpose of A by B
 *     (C~ = A^T B), hence the op(A) = A^T flag.
 *   - Paper Sec. 4: a contraction of two block-sparse tensors over 1..3 index sets
 *     is the sum over the contracted indices of the products of their elements.
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * project's design notes):
 *   - block elements are row-major (last index fastest);
 *   - block-norm filter: a block product A_ik * B_kj is kept iff
 *     ||A_ik||_F * ||B_kj||_F >= eps (equality kept; alpha does not enter);
 *   - pattern(C_out) = pattern(C_in) U {(i,j): some kept k}; no post-filter on C;
 *   - C_out = alpha * (sum over kept k ascending of A_ik B_kj) + beta * C_in, and
 *     with beta == 0 the values of C_in are never read;
 *   - stacks: one entry (a_off, b_off, c_off) per kept product, element offsets of
 *     the stored blocks, grouped into buckets by (m, n, k) sizes in lexicographic
 *     order and ordered by (i, j, k) block indices inside a bucket.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  OR_OK = 0,
  OR_ERR_INVALID_ARG = 1,
  OR_ERR_OUT_OF_RANGE = 2,
  OR_ERR_DUPLICATE_BLOCK = 3,
  OR_ERR_SHAPE_MISMATCH = 4,
  OR_ERR_OVERFLOW = 5,
  OR_ERR_ALLOC = 6
};

#define OR_I32_MAX 2147483647LL

/* ------------------------------------------------------------------------- */
/* matrices                                                                   */
/* ------------------------------------------------------------------------- */

/* A block-sparse matrix as handed in: block sizes per block row/column, the list
 * of present blocks in any order, and the data packed in canonical (row-major
 * over blocks, then row-major inside each block) order. */
typedef struct {
  int32_t nbr, nbc;
  const int32_t *rsz, *csz;
  int64_t nblocks;
  const int32_t *brow, *bcol;
  const double *data;
} or_matrix;

/* canonical form: blocks sorted by (row, col) with their element offsets */
typedef struct {
  int32_t nbr, nbc;
  const int32_t *rsz, *csz;
  int64_t nblocks;
  int32_t *row, *col;
  int64_t *off;
  int64_t nelem;
  const double *data;
} canon_t;

typedef struct {
  int64_t key;
  int64_t pos;
} kp_t;

static int cmp_kp(const void *a, const void *b) {
  const kp_t *x = (const kp_t *)a, *y = (const kp_t *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->pos < y->pos ? -1 : (x->pos > y->pos);
}

static void canon_free(canon_t *c) {
  free(c->row);
  free(c->col);
  free(c->off);
  memset(c, 0, sizeof(*c));
}

static int canonicalize(const or_matrix *m, canon_t *c) {
  memset(c, 0, sizeof(*c));
  if (!m || m->nbr < 0 || m->nbc < 0 || m->nblocks < 0) return OR_ERR_INVALID_ARG;
  if ((m->nbr && !m->rsz) || (m->nbc && !m->csz)) return OR_ERR_INVALID_ARG;
  if (m->nblocks && (!m->brow || !m->bcol)) return OR_ERR_INVALID_ARG;
  for (int32_t i = 0; i < m->nbr; ++i)
    if (m->rsz[i] <= 0) return OR_ERR_INVALID_ARG;
  for (int32_t j = 0; j < m->nbc; ++j)
    if (m->csz[j] <= 0) return OR_ERR_INVALID_ARG;
  int64_t n = m->nblocks;
  kp_t *kp = (kp_t *)malloc(sizeof(kp_t) * (size_t)(n ? n : 1));
  c->row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  c->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  c->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
  if (!kp || !c->row || !c->col || !c->off) {
    free(kp);
    canon_free(c);
    return OR_ERR_ALLOC;
  }
  for (int64_t b = 0; b < n; ++b) {
    if (m->brow[b] < 0 || m->brow[b] >= m->nbr || m->bcol[b] < 0 || m->bcol[b] >= m->nbc) {
      free(kp);
      canon_free(c);
      return OR_ERR_OUT_OF_RANGE;
    }
    kp[b].key = (int64_t)m->brow[b] * (int64_t)m->nbc + m->bcol[b];
    kp[b].pos = b;
  }
  qsort(kp, (size_t)n, sizeof(kp_t), cmp_kp);
  int64_t off = 0;
  for (int64_t b = 0; b < n; ++b) {
    if (b > 0 && kp[b].key == kp[b - 1].key) {
      free(kp);
      canon_free(c);
      return OR_ERR_DUPLICATE_BLOCK;
    }
    int32_t r = m->brow[kp[b].pos], q = m->bcol[kp[b].pos];
    c->row[b] = r;
    c->col[b] = q;
    c->off[b] = off;
    off += (int64_t)m->rsz[r] * m->csz[q];
  }
  free(kp);
  c->nbr = m->nbr;
  c->nbc = m->nbc;
  c->rsz = m->rsz;
  c->csz = m->csz;
  c->nblocks = n;
  c->nelem = off;
  c->data = m->data;
  if (n && !m->data) {
    canon_free(c);
    return OR_ERR_INVALID_ARG;
  }
  return OR_OK;
}

/* Frobenius norm of one block: sqrt of the sum of squares, taken in the block's
 * row-major element order. */
static double block_norm(const double *x, int64_t n) {
  double s = 0.0;
  for (int64_t e = 0; e < n; ++e) s += x[e] * x[e];
  return sqrt(s);
}

int or_block_norms(const or_matrix *m, double *norms_out) {
  canon_t c;
  int st = canonicalize(m, &c);
  if (st) return st;
  for (int64_t b = 0; b < c.nblocks; ++b)
    norms_out[b] = block_norm(c.data + c.off[b], (int64_t)c.rsz[c.row[b]] * c.csz[c.col[b]]);
  canon_free(&c);
  return OR_OK;
}

/* A block of op(X) as seen by the product: block indices (i, k) after the
 * optional transpose, the stored block it comes from, its shape after op. */
typedef struct {
  int32_t i, k;
  int64_t stored;
} opblk_t;

typedef struct {
  int32_t nr, nc;              /* block rows / cols of op(X) */
  const int32_t *rs, *cs;      /* block sizes of op(X) */
  int trans;
  int64_t n;
  opblk_t *blk;                /* sorted by (i, k) */
  int64_t *rowptr;             /* nr + 1 */
} opview_t;

static int cmp_opblk(const void *a, const void *b) {
  const opblk_t *x = (const opblk_t *)a, *y = (const opblk_t *)b;
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  if (x->k != y->k) return x->k < y->k ? -1 : 1;
  return 0;
}

static void opview_free(opview_t *v) {
  free(v->blk);
  free(v->rowptr);
  memset(v, 0, sizeof(*v));
}

static int make_opview(const canon_t *c, int trans, opview_t *v) {
  memset(v, 0, sizeof(*v));
  v->trans = trans;
  v->nr = trans ? c->nbc : c->nbr;
  v->nc = trans ? c->nbr : c->nbc;
  v->rs = trans ? c->csz : c->rsz;
  v->cs = trans ? c->rsz : c->csz;
  v->n = c->nblocks;
  v->blk = (opblk_t *)malloc(sizeof(opblk_t) * (size_t)(v->n ? v->n : 1));
  v->rowptr = (int64_t *)calloc((size_t)v->nr + 1, sizeof(int64_t));
  if (!v->blk || !v->rowptr) {
    opview_free(v);
    return OR_ERR_ALLOC;
  }
  for (int64_t b = 0; b < v->n; ++b) {
    v->blk[b].i = trans ? c->col[b] : c->row[b];
    v->blk[b].k = trans ? c->row[b] : c->col[b];
    v->blk[b].stored = b;
  }
  qsort(v->blk, (size_t)v->n, sizeof(opblk_t), cmp_opblk);
  for (int64_t b = 0; b < v->n; ++b) v->rowptr[v->blk[b].i + 1]++;
  for (int32_t r = 0; r < v->nr; ++r) v->rowptr[r + 1] += v->rowptr[r];
  return OR_OK;
}

/* element (p, l) of op(X) block `stored` whose op-shape is (rows x cols) */
static double op_elem(const canon_t *c, int trans, int64_t stored, int32_t rows, int32_t cols,
                      int32_t p, int32_t l) {
  const double *x = c->data + c->off[stored];
  return trans ? x[(int64_t)l * rows + p] : x[(int64_t)p * cols + l];
}

typedef struct {
  int32_t i, j, k;
  int32_t m, n, kk;
  int64_t sa, sb;
} triple_t;

static int cmp_triple_ijk(const void *a, const void *b) {
  const triple_t *x = (const triple_t *)a, *y = (const triple_t *)b;
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  if (x->j != y->j) return x->j < y->j ? -1 : 1;
  if (x->k != y->k) return x->k < y->k ? -1 : 1;
  return 0;
}

static int cmp_triple_bucket(const void *a, const void *b) {
  const triple_t *x = (const triple_t *)a, *y = (const triple_t *)b;
  if (x->m != y->m) return x->m < y->m ? -1 : 1;
  if (x->n != y->n) return x->n < y->n ? -1 : 1;
  if (x->kk != y->kk) return x->kk < y->kk ? -1 : 1;
  return cmp_triple_ijk(a, b);
}

typedef struct {
  int32_t i, j;
} ij_t;

static int cmp_ij(const void *a, const void *b) {
  const ij_t *x = (const ij_t *)a, *y = (const ij_t *)b;
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  if (x->j != y->j) return x->j < y->j ? -1 : 1;
  return 0;
}

/* result of a multiply: C_out pattern + data, stacks and counters */
typedef struct {
  int32_t nbr, nbc;
  int64_t nblocks, nelem;
  int32_t *brow, *bcol;
  int64_t *boff;
  double *data;
  int64_t nstack;
  int32_t nbuckets;
  int32_t *mnk;          /* nbuckets * 3 */
  int64_t *bucket_ptr;   /* nbuckets + 1 */
  int32_t *a_off, *b_off, *c_off;
  int64_t ncandidates, nfiltered;
  double flops;
} or_result;

void or_result_free(or_result *r) {
  if (!r) return;
  free(r->brow);
  free(r->bcol);
  free(r->boff);
  free(r->data);
  free(r->mnk);
  free(r->bucket_ptr);
  free(r->a_off);
  free(r->b_off);
  free(r->c_off);
  free(r);
}

void or_result_sizes(const or_result *r, int64_t *sizes /* [6] */) {
  sizes[0] = r->nblocks;
  sizes[1] = r->nelem;
  sizes[2] = r->nstack;
  sizes[3] = r->nbuckets;
  sizes[4] = r->ncandidates;
  sizes[5] = r->nfiltered;
}

double or_result_flops(const or_result *r) { return r->flops; }

void or_result_get(const or_result *r, int32_t *brow, int32_t *bcol, int64_t *boff, double *data,
                   int32_t *mnk, int64_t *bucket_ptr, int32_t *a_off, int32_t *b_off,
                   int32_t *c_off) {
  if (brow) memcpy(brow, r->brow, sizeof(int32_t) * (size_t)r->nblocks);
  if (bcol) memcpy(bcol, r->bcol, sizeof(int32_t) * (size_t)r->nblocks);
  if (boff) memcpy(boff, r->boff, sizeof(int64_t) * (size_t)r->nblocks);
  if (data) memcpy(data, r->data, sizeof(double) * (size_t)r->nelem);
  if (mnk) memcpy(mnk, r->mnk, sizeof(int32_t) * 3 * (size_t)r->nbuckets);
  if (bucket_ptr) memcpy(bucket_ptr, r->bucket_ptr, sizeof(int64_t) * ((size_t)r->nbuckets + 1));
  if (a_off) memcpy(a_off, r->a_off, sizeof(int32_t) * (size_t)r->nstack);
  if (b_off) memcpy(b_off, r->b_off, sizeof(int32_t) * (size_t)r->nstack);
  if (c_off) memcpy(c_off, r->c_off, sizeof(int32_t) * (size_t)r->nstack);
}

/* find block (i, j) in a canonical matrix; -1 if absent */
static int64_t find_block(const canon_t *c, int32_t i, int32_t j) {
  int64_t lo = 0, hi = c->nblocks;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (c->row[mid] < i || (c->row[mid] == i && c->col[mid] < j))
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < c->nblocks && c->row[lo] == i && c->col[lo] == j) return lo;
  return -1;
}

/* common set-up of a multiply: canonical inputs, op views, shape checks */
typedef struct {
  canon_t A, B, Ci;
  int has_cin;
  opview_t oa, ob;
  double *na, *nb;
} mulsetup_t;

static void mulsetup_free(mulsetup_t *s) {
  canon_free(&s->A);
  canon_free(&s->B);
  canon_free(&s->Ci);
  opview_free(&s->oa);
  opview_free(&s->ob);
  free(s->na);
  free(s->nb);
  memset(s, 0, sizeof(*s));
}

static int mulsetup(char transa, char transb, const or_matrix *A, const or_matrix *B,
                    const or_matrix *Cin, mulsetup_t *s) {
  memset(s, 0, sizeof(*s));
  int ta, tb;
  if (transa == 'N' || transa == 'n') ta = 0;
  else if (transa == 'T' || transa == 't') ta = 1;
  else return OR_ERR_INVALID_ARG;
  if (transb == 'N' || transb == 'n') tb = 0;
  else if (transb == 'T' || transb == 't') tb = 1;
  else return OR_ERR_INVALID_ARG;
  int st = canonicalize(A, &s->A);
  if (!st) st = canonicalize(B, &s->B);
  if (!st && Cin) {
    st = canonicalize(Cin, &s->Ci);
    s->has_cin = 1;
  }
  if (!st) st = make_opview(&s->A, ta, &s->oa);
  if (!st) st = make_opview(&s->B, tb, &s->ob);
  if (st) {
    mulsetup_free(s);
    return st;
  }
  /* inner dimension: block columns of op(A) must be the block rows of op(B) */
  if (s->oa.nc != s->ob.nr) st = OR_ERR_SHAPE_MISMATCH;
  for (int32_t k = 0; !st && k < s->oa.nc; ++k)
    if (s->oa.cs[k] != s->ob.rs[k]) st = OR_ERR_SHAPE_MISMATCH;
  if (!st && s->has_cin) {
    if (s->Ci.nbr != s->oa.nr || s->Ci.nbc != s->ob.nc) st = OR_ERR_SHAPE_MISMATCH;
    for (int32_t i = 0; !st && i < s->oa.nr; ++i)
      if (s->Ci.rsz[i] != s->oa.rs[i]) st = OR_ERR_SHAPE_MISMATCH;
    for (int32_t j = 0; !st && j < s->ob.nc; ++j)
      if (s->Ci.csz[j] != s->ob.cs[j]) st = OR_ERR_SHAPE_MISMATCH;
  }
  if (!st && (s->A.nelem > OR_I32_MAX || s->B.nelem > OR_I32_MAX)) st = OR_ERR_OVERFLOW;
  if (!st) {
    s->na = (double *)malloc(sizeof(double) * (size_t)(s->A.nblocks ? s->A.nblocks : 1));
    s->nb = (double *)malloc(sizeof(double) * (size_t)(s->B.nblocks ? s->B.nblocks : 1));
    if (!s->na || !s->nb) st = OR_ERR_ALLOC;
  }
  if (st) {
    mulsetup_free(s);
    return st;
  }
  for (int64_t b = 0; b < s->A.nblocks; ++b)
    s->na[b] = block_norm(s->A.data + s->A.off[b],
                          (int64_t)s->A.rsz[s->A.row[b]] * s->A.csz[s->A.col[b]]);
  for (int64_t b = 0; b < s->B.nblocks; ++b)
    s->nb[b] = block_norm(s->B.data + s->B.off[b],
                          (int64_t)s->B.rsz[s->B.row[b]] * s->B.csz[s->B.col[b]]);
  return OR_OK;
}

/* C_out = alpha * op(A) * op(B) + beta * C_in with the block-norm filter eps. */
int or_multiply(char transa, char transb, const or_matrix *A, const or_matrix *B,
                const or_matrix *Cin, double alpha, double beta, double eps, or_result **out) {
  *out = NULL;
  if (!(eps >= 0.0)) return OR_ERR_INVALID_ARG;
  mulsetup_t s;
  int st = mulsetup(transa, transb, A, B, Cin, &s);
  if (st) return st;
  opview_t *oa = &s.oa, *ob = &s.ob;

  /* 1. all kept (i, k, j) triples: loop over the row blocks of op(A), then over
   *    the blocks of op(B) in the matching row k (paper Sec. 2). */
  int64_t cap = 1024, nt = 0, ncand = 0, nfilt = 0;
  triple_t *t = (triple_t *)malloc(sizeof(triple_t) * (size_t)cap);
  if (!t) {
    mulsetup_free(&s);
    return OR_ERR_ALLOC;
  }
  for (int64_t a = 0; a < oa->n; ++a) {
    int32_t i = oa->blk[a].i, k = oa->blk[a].k;
    for (int64_t b = ob->rowptr[k]; b < ob->rowptr[k + 1]; ++b) {
      ++ncand;
      double pn = s.na[oa->blk[a].stored] * s.nb[ob->blk[b].stored];
      if (!(pn >= eps)) {
        ++nfilt;
        continue;
      }
      if (nt == cap) {
        cap *= 2;
        triple_t *t2 = (triple_t *)realloc(t, sizeof(triple_t) * (size_t)cap);
        if (!t2) {
          free(t);
          mulsetup_free(&s);
          return OR_ERR_ALLOC;
        }
        t = t2;
      }
      t[nt].i = i;
      t[nt].j = ob->blk[b].k;
      t[nt].k = k;
      t[nt].m = oa->rs[i];
      t[nt].n = ob->cs[ob->blk[b].k];
      t[nt].kk = oa->cs[k];
      t[nt].sa = oa->blk[a].stored;
      t[nt].sb = ob->blk[b].stored;
      ++nt;
    }
  }

  /* 2. pattern of C_out: pattern(C_in) united with every (i, j) of a kept triple */
  int64_t nij = nt + (s.has_cin ? s.Ci.nblocks : 0);
  ij_t *ij = (ij_t *)malloc(sizeof(ij_t) * (size_t)(nij ? nij : 1));
  or_result *r = (or_result *)calloc(1, sizeof(or_result));
  if (!ij || !r) {
    free(t);
    free(ij);
    free(r);
    mulsetup_free(&s);
    return OR_ERR_ALLOC;
  }
  for (int64_t e = 0; e < nt; ++e) {
    ij[e].i = t[e].i;
    ij[e].j = t[e].j;
  }
  for (int64_t e = 0; s.has_cin && e < s.Ci.nblocks; ++e) {
    ij[nt + e].i = s.Ci.row[e];
    ij[nt + e].j = s.Ci.col[e];
  }
  qsort(ij, (size_t)nij, sizeof(ij_t), cmp_ij);
  int64_t nc = 0;
  for (int64_t e = 0; e < nij; ++e)
    if (nc == 0 || cmp_ij(&ij[e], &ij[nc - 1]) != 0) ij[nc++] = ij[e];

  r->nbr = oa->nr;
  r->nbc = ob->nc;
  r->nblocks = nc;
  r->brow = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));
  r->bcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc ? nc : 1));
  r->boff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc ? nc : 1));
  if (!r->brow || !r->bcol || !r->boff) st = OR_ERR_ALLOC;
  int64_t off = 0;
  for (int64_t e = 0; !st && e < nc; ++e) {
    r->brow[e] = ij[e].i;
    r->bcol[e] = ij[e].j;
    r->boff[e] = off;
    off += (int64_t)oa->rs[ij[e].i] * ob->cs[ij[e].j];
  }
  free(ij);
  r->nelem = off;
  if (!st && off > OR_I32_MAX) st = OR_ERR_OVERFLOW;
  if (!st) {
    r->data = (double *)calloc((size_t)(off ? off : 1), sizeof(double));
    if (!r->data) st = OR_ERR_ALLOC;
  }
  canon_t cc;
  memset(&cc, 0, sizeof(cc));
  cc.nbr = r->nbr;
  cc.nbc = r->nbc;
  cc.nblocks = nc;
  cc.row = r->brow;
  cc.col = r->bcol;
  cc.off = r->boff;

  /* 3. values: acc(i,j) = sum over kept k ascending of A_ik * B_kj, each block
   *    product element being sum_l a[p][l] * b[l][q] with l ascending; then
   *    C_out = alpha * acc + beta * C_in (C_in unread when beta == 0). */
  if (!st) {
    qsort(t, (size_t)nt, sizeof(triple_t), cmp_triple_ijk);
    for (int64_t e = 0; e < nt; ++e) {
      int64_t cb = find_block(&cc, t[e].i, t[e].j);
      double *c = r->data + r->boff[cb];
      int32_t m = t[e].m, n = t[e].n, kk = t[e].kk;
      for (int32_t p = 0; p < m; ++p)
        for (int32_t q = 0; q < n; ++q) {
          double dot = 0.0;
          for (int32_t l = 0; l < kk; ++l)
            dot += op_elem(&s.A, oa->trans, t[e].sa, m, kk, p, l) *
                   op_elem(&s.B, ob->trans, t[e].sb, kk, n, l, q);
          c[(int64_t)p * n + q] += dot;
        }
    }
    for (int64_t cb = 0; cb < nc; ++cb) {
      int64_t len = (int64_t)oa->rs[r->brow[cb]] * ob->cs[r->bcol[cb]];
      double *c = r->data + r->boff[cb];
      int64_t ib = (s.has_cin && beta != 0.0) ? find_block(&s.Ci, r->brow[cb], r->bcol[cb]) : -1;
      for (int64_t e = 0; e < len; ++e) {
        double v = alpha * c[e];
        if (ib >= 0) v += beta * s.Ci.data[s.Ci.off[ib] + e];
        c[e] = v;
      }
    }
  }

  /* 4. stacks: buckets by (m, n, k) sizes, (i, j, k) order inside a bucket */
  if (!st) {
    qsort(t, (size_t)nt, sizeof(triple_t), cmp_triple_bucket);
    r->nstack = nt;
    r->a_off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    r->b_off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    r->c_off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    r->mnk = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(nt ? nt : 1));
    r->bucket_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt + 1));
    if (!r->a_off || !r->b_off || !r->c_off || !r->mnk || !r->bucket_ptr) st = OR_ERR_ALLOC;
  }
  if (!st) {
    int32_t nb = 0;
    double flops = 0.0;
    for (int64_t e = 0; e < nt; ++e) {
      if (e == 0 || t[e].m != t[e - 1].m || t[e].n != t[e - 1].n || t[e].kk != t[e - 1].kk) {
        r->mnk[3 * nb + 0] = t[e].m;
        r->mnk[3 * nb + 1] = t[e].n;
        r->mnk[3 * nb + 2] = t[e].kk;
        r->bucket_ptr[nb] = e;
        ++nb;
      }
      r->a_off[e] = (int32_t)s.A.off[t[e].sa];
      r->b_off[e] = (int32_t)s.B.off[t[e].sb];
      r->c_off[e] = (int32_t)r->boff[find_block(&cc, t[e].i, t[e].j)];
      flops += 2.0 * t[e].m * t[e].n * t[e].kk;
    }
    r->bucket_ptr[nb] = nt;
    r->nbuckets = nb;
    r->flops = flops;
    r->ncandidates = ncand;
    r->nfiltered = nfilt;
  }
  free(t);
  mulsetup_free(&s);
  if (st) {
    or_result_free(r);
    return st;
  }
  *out = r;
  return OR_OK;
}

/* Values of selected blocks (i, j) of C_out only, from the same definition:
 * for each requested block, sum over k ascending of the kept products, then
 * alpha * acc + beta * C_in.  Blocks outside pattern(C_out) come back as zeros and
 * present[e] = 0.  out is packed in request order, each block m x n row-major. */
int or_multiply_sample(char transa, char transb, const or_matrix *A, const or_matrix *B,
                       const or_matrix *Cin, double alpha, double beta, double eps,
                       int64_t nreq, const int32_t *ri, const int32_t *rj, double *out,
                       int8_t *present) {
  if (!(eps >= 0.0)) return OR_ERR_INVALID_ARG;
  mulsetup_t s;
  int st = mulsetup(transa, transb, A, B, Cin, &s);
  if (st) return st;
  opview_t *oa = &s.oa, *ob = &s.ob;
  int64_t pos = 0;
  for (int64_t e = 0; e < nreq; ++e) {
    int32_t i = ri[e], j = rj[e];
    if (i < 0 || i >= oa->nr || j < 0 || j >= ob->nc) {
      mulsetup_free(&s);
      return OR_ERR_OUT_OF_RANGE;
    }
    int32_t m = oa->rs[i], n = ob->cs[j];
    double *c = out + pos;
    for (int64_t x = 0; x < (int64_t)m * n; ++x) c[x] = 0.0;
    int any = 0;
    for (int64_t a = oa->rowptr[i]; a < oa->rowptr[i + 1]; ++a) {
      int32_t k = oa->blk[a].k, kk = oa->cs[k];
      for (int64_t b = ob->rowptr[k]; b < ob->rowptr[k + 1]; ++b) {
        if (ob->blk[b].k != j) continue;
        double pn = s.na[oa->blk[a].stored] * s.nb[ob->blk[b].stored];
        if (!(pn >= eps)) continue;
        any = 1;
        for (int32_t p = 0; p < m; ++p)
          for (int32_t q = 0; q < n; ++q) {
            double dot = 0.0;
            for (int32_t l = 0; l < kk; ++l)
              dot += op_elem(&s.A, oa->trans, oa->blk[a].stored, m, kk, p, l) *
                     op_elem(&s.B, ob->trans, ob->blk[b].stored, kk, n, l, q);
            c[(int64_t)p * n + q] += dot;
          }
      }
    }
    int64_t ib = s.has_cin ? find_block(&s.Ci, i, j) : -1;
    if (ib >= 0) any = 1;
    for (int64_t x = 0; x < (int64_t)m * n; ++x) {
      double v = alpha * c[x];
      if (ib >= 0 && beta != 0.0) v += beta * s.Ci.data[s.Ci.off[ib] + x];
      c[x] = v;
    }
    if (present) present[e] = (int8_t)any;
    pos += (int64_t)m * n;
  }
  mulsetup_free(&s);
  return OR_OK;
}

/* Adjoint of the computed function C_out = alpha op(A) op(B) + beta C_in with the
 * filter decisions held fixed: given dC on pattern(C_out),
 *   dop(A)_ik = alpha * sum_{j: (i,k,j) kept} dC_ij op(B)_kj^T   on pattern(A),
 *   dop(B)_kj = alpha * sum_{i: (i,k,j) kept} op(A)_ik^T dC_ij   on pattern(B),
 *   dC_in = beta * dC                                            on pattern(C_in),
 * returned in the stored layout of A, B and C_in (a transposed operand gets the
 * transpose of its op-gradient).  dC is packed in the canonical C_out order that
 * or_multiply returns. */
int or_multiply_adjoint(char transa, char transb, const or_matrix *A, const or_matrix *B,
                        const or_matrix *Cin, double alpha, double beta, double eps,
                        const double *dC, double *dA, double *dB, double *dCin) {
  or_result *res = NULL;
  int st = or_multiply(transa, transb, A, B, Cin, alpha, beta, eps, &res);
  if (st) return st;
  mulsetup_t s;
  st = mulsetup(transa, transb, A, B, Cin, &s);
  if (st) {
    or_result_free(res);
    return st;
  }
  opview_t *oa = &s.oa, *ob = &s.ob;
  canon_t cc;
  memset(&cc, 0, sizeof(cc));
  cc.nbr = res->nbr;
  cc.nbc = res->nbc;
  cc.nblocks = res->nblocks;
  cc.row = res->brow;
  cc.col = res->bcol;
  cc.off = res->boff;
  memset(dA, 0, sizeof(double) * (size_t)s.A.nelem);
  memset(dB, 0, sizeof(double) * (size_t)s.B.nelem);
  for (int64_t a = 0; a < oa->n; ++a) {
    int32_t i = oa->blk[a].i, k = oa->blk[a].k, m = oa->rs[i], kk = oa->cs[k];
    int64_t sa = oa->blk[a].stored;
    for (int64_t b = ob->rowptr[k]; b < ob->rowptr[k + 1]; ++b) {
      int64_t sb = ob->blk[b].stored;
      if (!(s.na[sa] * s.nb[sb] >= eps)) continue;
      int32_t j = ob->blk[b].k, n = ob->cs[j];
      const double *g = dC + res->boff[find_block(&cc, i, j)];
      /* dop(A)[p][l] += alpha * sum_q g[p][q] * op(B)[l][q] */
      for (int32_t p = 0; p < m; ++p)
        for (int32_t l = 0; l < kk; ++l) {
          double dot = 0.0;
          for (int32_t q = 0; q < n; ++q)
            dot += g[(int64_t)p * n + q] * op_elem(&s.B, ob->trans, sb, kk, n, l, q);
          int64_t idx = oa->trans ? (int64_t)l * m + p : (int64_t)p * kk + l;
          dA[s.A.off[sa] + idx] += alpha * dot;
        }
      /* dop(B)[l][q] += alpha * sum_p op(A)[p][l] * g[p][q] */
      for (int32_t l = 0; l < kk; ++l)
        for (int32_t q = 0; q < n; ++q) {
          double dot = 0.0;
          for (int32_t p = 0; p < m; ++p)
            dot += op_elem(&s.A, oa->trans, sa, m, kk, p, l) * g[(int64_t)p * n + q];
          int64_t idx = ob->trans ? (int64_t)q * kk + l : (int64_t)l * n + q;
          dB[s.B.off[sb] + idx] += alpha * dot;
        }
    }
  }
  if (s.has_cin && dCin) {
    for (int64_t cb = 0; cb < s.Ci.nblocks; ++cb) {
      int64_t ob_ = find_block(&cc, s.Ci.row[cb], s.Ci.col[cb]);
      int64_t len = (int64_t)s.Ci.rsz[s.Ci.row[cb]] * s.Ci.csz[s.Ci.col[cb]];
      for (int64_t e = 0; e < len; ++e) dCin[s.Ci.off[cb] + e] = beta * dC[res->boff[ob_] + e];
    }
  }
  mulsetup_free(&s);
  or_result_free(res);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* tensors (paper Sec. 4)                                                     */
/* ------------------------------------------------------------------------- */

#define OR_MAXRANK 8

/* A block-sparse tensor: per-mode block sizes (bsz holds the sizes of mode 0,
 * then mode 1, ...), block index tuples (nblocks x rank, any order) and data
 * packed in lexicographic tuple order, each block row-major (last mode fastest). */
typedef struct {
  int32_t rank;
  const int32_t *nblk;
  const int32_t *bsz;
  int64_t nblocks;
  const int32_t *idx;
  const double *data;
} or_tensor;

typedef struct {
  int32_t rank;
  int32_t nblk[OR_MAXRANK];
  const int32_t *sz[OR_MAXRANK];
  int64_t nblocks;
  int32_t *idx;   /* canonical order, nblocks x rank */
  int64_t *off;
  int64_t nelem;
  const double *data;
} tcanon_t;

static const int32_t *g_sort_idx;
static int32_t g_sort_rank;

static int cmp_tuple_pos(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  for (int32_t d = 0; d < g_sort_rank; ++d) {
    int32_t u = g_sort_idx[x * g_sort_rank + d], v = g_sort_idx[y * g_sort_rank + d];
    if (u != v) return u < v ? -1 : 1;
  }
  return 0;
}

static void tcanon_free(tcanon_t *c) {
  free(c->idx);
  free(c->off);
  memset(c, 0, sizeof(*c));
}

static int64_t tblock_len(const tcanon_t *c, const int32_t *tup) {
  int64_t len = 1;
  for (int32_t d = 0; d < c->rank; ++d) len *= c->sz[d][tup[d]];
  return len;
}

static int tcanonicalize(const or_tensor *t, tcanon_t *c) {
  memset(c, 0, sizeof(*c));
  if (!t || t->rank < 1 || t->rank > OR_MAXRANK || t->nblocks < 0) return OR_ERR_INVALID_ARG;
  c->rank = t->rank;
  int64_t so = 0;
  for (int32_t d = 0; d < t->rank; ++d) {
    if (t->nblk[d] < 0) return OR_ERR_INVALID_ARG;
    c->nblk[d] = t->nblk[d];
    c->sz[d] = t->bsz + so;
    for (int32_t b = 0; b < t->nblk[d]; ++b)
      if (c->sz[d][b] <= 0) return OR_ERR_INVALID_ARG;
    so += t->nblk[d];
  }
  int64_t n = t->nblocks;
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
  c->idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1) * (size_t)t->rank);
  c->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
  if (!perm || !c->idx || !c->off) {
    free(perm);
    tcanon_free(c);
    return OR_ERR_ALLOC;
  }
  for (int64_t b = 0; b < n; ++b) {
    perm[b] = b;
    for (int32_t d = 0; d < t->rank; ++d) {
      int32_t v = t->idx[b * t->rank + d];
      if (v < 0 || v >= t->nblk[d]) {
        free(perm);
        tcanon_free(c);
        return OR_ERR_OUT_OF_RANGE;
      }
    }
  }
  g_sort_idx = t->idx;
  g_sort_rank = t->rank;
  qsort(perm, (size_t)n, sizeof(int64_t), cmp_tuple_pos);
  int64_t off = 0;
  for (int64_t b = 0; b < n; ++b) {
    if (b > 0 && cmp_tuple_pos(&perm[b], &perm[b - 1]) == 0) {
      free(perm);
      tcanon_free(c);
      return OR_ERR_DUPLICATE_BLOCK;
    }
    memcpy(c->idx + b * t->rank, t->idx + perm[b] * t->rank, sizeof(int32_t) * (size_t)t->rank);
    c->off[b] = off;
    off += tblock_len(c, c->idx + b * t->rank);
  }
  free(perm);
  c->nblocks = n;
  c->nelem = off;
  c->data = t->data;
  if (n && !t->data) {
    tcanon_free(c);
    return OR_ERR_INVALID_ARG;
  }
  return OR_OK;
}

static int64_t tfind(const tcanon_t *c, const int32_t *tup) {
  int64_t lo = 0, hi = c->nblocks;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2, d;
    int cmp = 0;
    for (d = 0; d < c->rank && !cmp; ++d) {
      int32_t u = c->idx[mid * c->rank + d];
      cmp = (u < tup[d]) ? -1 : (u > tup[d]);
    }
    if (cmp < 0)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < c->nblocks && memcmp(c->idx + lo * c->rank, tup, sizeof(int32_t) * (size_t)c->rank) == 0)
    return lo;
  return -1;
}

/* row-major strides of the elements of one block */
static void block_strides(const tcanon_t *c, const int32_t *tup, int64_t *stride) {
  int64_t s = 1;
  for (int32_t d = c->rank - 1; d >= 0; --d) {
    stride[d] = s;
    s *= c->sz[d][tup[d]];
  }
}

typedef struct {
  int32_t rank;
  int32_t nblk[OR_MAXRANK];
  int32_t *bsz;       /* concatenated per-mode sizes */
  int64_t nblocks;
  int32_t *idx;       /* canonical order */
  int64_t *off;
  int64_t nelem;
  double *data;
  int64_t npairs, nfiltered;
  double flops;
} or_tresult;

void or_tresult_free(or_tresult *r) {
  if (!r) return;
  free(r->bsz);
  free(r->idx);
  free(r->off);
  free(r->data);
  free(r);
}

void or_tresult_sizes(const or_tresult *r, int64_t *sizes /* [5] */) {
  sizes[0] = r->rank;
  sizes[1] = r->nblocks;
  sizes[2] = r->nelem;
  sizes[3] = r->npairs;
  sizes[4] = r->nfiltered;
}

double or_tresult_flops(const or_tresult *r) { return r->flops; }

void or_tresult_get(const or_tresult *r, int32_t *idx, int64_t *off, double *data) {
  if (idx) memcpy(idx, r->idx, sizeof(int32_t) * (size_t)r->nblocks * (size_t)r->rank);
  if (off) memcpy(off, r->off, sizeof(int64_t) * (size_t)r->nblocks);
  if (data) memcpy(data, r->data, sizeof(double) * (size_t)r->nelem);
}

/* contraction specification after validation */
typedef struct {
  tcanon_t t1, t2, ri;
  int has_rin;
  int32_t nc, nf1, nf2, rrank;
  int32_t c1[OR_MAXRANK], c2[OR_MAXRANK], f1[OR_MAXRANK], f2[OR_MAXRANK];
  int32_t ro[OR_MAXRANK];      /* result mode r takes free slot ro[r] of (f1..., f2...) */
  double *n1, *n2;
} cset_t;

static void cset_free(cset_t *s) {
  tcanon_free(&s->t1);
  tcanon_free(&s->t2);
  tcanon_free(&s->ri);
  free(s->n1);
  free(s->n2);
  memset(s, 0, sizeof(*s));
}

/* block size of free slot f of the result for the block pair (b1, b2) */
static int32_t free_slot_mode_size(const cset_t *s, int32_t slot, int32_t bi) {
  if (slot < s->nf1) return s->t1.sz[s->f1[slot]][bi];
  return s->t2.sz[s->f2[slot - s->nf1]][bi];
}

static int cset_make(const or_tensor *T1, const or_tensor *T2, int32_t nc, const int32_t *c1,
                     const int32_t *c2, int32_t nf1, const int32_t *f1, int32_t nf2,
                     const int32_t *f2, const int32_t *result_order, const or_tensor *Rin,
                     cset_t *s) {
  memset(s, 0, sizeof(*s));
  int st = tcanonicalize(T1, &s->t1);
  if (!st) st = tcanonicalize(T2, &s->t2);
  if (!st && Rin) {
    st = tcanonicalize(Rin, &s->ri);
    s->has_rin = 1;
  }
  if (st) {
    cset_free(s);
    return st;
  }
  int32_t d1 = s->t1.rank, d2 = s->t2.rank;
  if (nc < 1 || nc > 3 || nf1 < 0 || nf2 < 0 || nc + nf1 != d1 || nc + nf2 != d2 ||
      nf1 + nf2 < 1) {
    cset_free(s);
    return OR_ERR_INVALID_ARG;
  }
  /* each mode of T1 (T2) is listed exactly once in c1 + f1 (c2 + f2) */
  int32_t seen1[OR_MAXRANK] = {0}, seen2[OR_MAXRANK] = {0}, seenr[2 * OR_MAXRANK] = {0};
  for (int32_t x = 0; x < nc; ++x) {
    if (c1[x] < 0 || c1[x] >= d1 || c2[x] < 0 || c2[x] >= d2 || seen1[c1[x]]++ || seen2[c2[x]]++) {
      cset_free(s);
      return OR_ERR_INVALID_ARG;
    }
    s->c1[x] = c1[x];
    s->c2[x] = c2[x];
  }
  for (int32_t x = 0; x < nf1; ++x) {
    if (f1[x] < 0 || f1[x] >= d1 || seen1[f1[x]]++) {
      cset_free(s);
      return OR_ERR_INVALID_ARG;
    }
    s->f1[x] = f1[x];
  }
  for (int32_t x = 0; x < nf2; ++x) {
    if (f2[x] < 0 || f2[x] >= d2 || seen2[f2[x]]++) {
      cset_free(s);
      return OR_ERR_INVALID_ARG;
    }
    s->f2[x] = f2[x];
  }
  s->nc = nc;
  s->nf1 = nf1;
  s->nf2 = nf2;
  s->rrank = nf1 + nf2;
  for (int32_t r = 0; r < s->rrank; ++r) {
    int32_t v = result_order ? result_order[r] : r;
    if (v < 0 || v >= s->rrank || seenr[v]++) {
      cset_free(s);
      return OR_ERR_INVALID_ARG;
    }
    s->ro[r] = v;
  }
  /* contracted modes must have identical block sizes mode by mode */
  for (int32_t x = 0; x < nc; ++x) {
    int32_t a = c1[x], b = c2[x];
    if (s->t1.nblk[a] != s->t2.nblk[b]) {
      cset_free(s);
      return OR_ERR_SHAPE_MISMATCH;
    }
    for (int32_t q = 0; q < s->t1.nblk[a]; ++q)
      if (s->t1.sz[a][q] != s->t2.sz[b][q]) {
        cset_free(s);
        return OR_ERR_SHAPE_MISMATCH;
      }
  }
  if (s->has_rin) {
    if (s->ri.rank != s->rrank) {
      cset_free(s);
      return OR_ERR_SHAPE_MISMATCH;
    }
    for (int32_t r = 0; r < s->rrank; ++r) {
      int32_t slot = s->ro[r];
      int32_t mode_nblk = slot < nf1 ? s->t1.nblk[f1[slot]] : s->t2.nblk[f2[slot - nf1]];
      if (s->ri.nblk[r] != mode_nblk) {
        cset_free(s);
        return OR_ERR_SHAPE_MISMATCH;
      }
      for (int32_t q = 0; q < mode_nblk; ++q)
        if (s->ri.sz[r][q] != free_slot_mode_size(s, slot, q)) {
          cset_free(s);
          return OR_ERR_SHAPE_MISMATCH;
        }
    }
  }
  s->n1 = (double *)malloc(sizeof(double) * (size_t)(s->t1.nblocks ? s->t1.nblocks : 1));
  s->n2 = (double *)malloc(sizeof(double) * (size_t)(s->t2.nblocks ? s->t2.nblocks : 1));
  if (!s->n1 || !s->n2) {
    cset_free(s);
    return OR_ERR_ALLOC;
  }
  for (int64_t b = 0; b < s->t1.nblocks; ++b)
    s->n1[b] = block_norm(s->t1.data + s->t1.off[b], tblock_len(&s->t1, s->t1.idx + b * d1));
  for (int64_t b = 0; b < s->t2.nblocks; ++b)
    s->n2[b] = block_norm(s->t2.data + s->t2.off[b], tblock_len(&s->t2, s->t2.idx + b * d2));
  return OR_OK;
}

/* do blocks b1 of T1 and b2 of T2 agree on every contracted block index? */
static int pair_matches(const cset_t *s, int64_t b1, int64_t b2) {
  for (int32_t x = 0; x < s->nc; ++x)
    if (s->t1.idx[b1 * s->t1.rank + s->c1[x]] != s->t2.idx[b2 * s->t2.rank + s->c2[x]]) return 0;
  return 1;
}

/* block tuple of the result for the pair (b1, b2) */
static void result_tuple(const cset_t *s, int64_t b1, int64_t b2, int32_t *tup) {
  int32_t slots[2 * OR_MAXRANK];
  for (int32_t x = 0; x < s->nf1; ++x) slots[x] = s->t1.idx[b1 * s->t1.rank + s->f1[x]];
  for (int32_t x = 0; x < s->nf2; ++x) slots[s->nf1 + x] = s->t2.idx[b2 * s->t2.rank + s->f2[x]];
  for (int32_t r = 0; r < s->rrank; ++r) tup[r] = slots[s->ro[r]];
}

/* the contraction of one block pair, written as the explicit index sum:
 * mode is one of: 0 = R[u,v] += sum_x T1[u,x] T2[x,v] (into out = R block),
 *                 1 = dT1[u,x] += sum_v dR[u,v] T2[x,v] (out = dT1 block, g = dR block),
 *                 2 = dT2[x,v] += sum_u T1[u,x] dR[u,v] (out = dT2 block, g = dR block).
 * u runs over the free element indices of T1, v over those of T2, x over the
 * contracted element indices; all as odometers over the listed modes. */
static void pair_kernel(const cset_t *s, int64_t b1, int64_t b2, int mode, const double *g,
                        double *out, double scale) {
  const int32_t *t1 = s->t1.idx + b1 * s->t1.rank, *t2 = s->t2.idx + b2 * s->t2.rank;
  int64_t st1[OR_MAXRANK], st2[OR_MAXRANK], str[2 * OR_MAXRANK];
  block_strides(&s->t1, t1, st1);
  block_strides(&s->t2, t2, st2);
  /* element extents of u (free of T1), v (free of T2), x (contracted) */
  int32_t eu[OR_MAXRANK], ev[OR_MAXRANK], ex[OR_MAXRANK];
  int64_t nu = 1, nv = 1, nx = 1;
  for (int32_t a = 0; a < s->nf1; ++a) nu *= (eu[a] = s->t1.sz[s->f1[a]][t1[s->f1[a]]]);
  for (int32_t a = 0; a < s->nf2; ++a) nv *= (ev[a] = s->t2.sz[s->f2[a]][t2[s->f2[a]]]);
  for (int32_t a = 0; a < s->nc; ++a) nx *= (ex[a] = s->t1.sz[s->c1[a]][t1[s->c1[a]]]);
  /* strides of the result block for each free slot */
  int32_t rt[2 * OR_MAXRANK], rsz[2 * OR_MAXRANK];
  result_tuple(s, b1, b2, rt);
  for (int32_t r = 0; r < s->rrank; ++r) rsz[r] = free_slot_mode_size(s, s->ro[r], rt[r]);
  {
    int64_t acc = 1;
    int64_t rstride[2 * OR_MAXRANK];
    for (int32_t r = s->rrank - 1; r >= 0; --r) {
      rstride[r] = acc;
      acc *= rsz[r];
    }
    for (int32_t r = 0; r < s->rrank; ++r) str[s->ro[r]] = rstride[r];
  }
  const double *d1 = s->t1.data + s->t1.off[b1], *d2 = s->t2.data + s->t2.off[b2];
  int32_t iu[OR_MAXRANK], iv[OR_MAXRANK], ix[OR_MAXRANK];
  memset(iu, 0, sizeof(iu));
  for (int64_t u = 0; u < nu; ++u) {
    memset(iv, 0, sizeof(iv));
    for (int64_t v = 0; v < nv; ++v) {
      int64_t o1u = 0, o2v = 0, orv = 0;
      for (int32_t a = 0; a < s->nf1; ++a) {
        o1u += st1[s->f1[a]] * iu[a];
        orv += str[a] * iu[a];
      }
      for (int32_t a = 0; a < s->nf2; ++a) {
        o2v += st2[s->f2[a]] * iv[a];
        orv += str[s->nf1 + a] * iv[a];
      }
      if (mode == 0) {
        double dot = 0.0;
        memset(ix, 0, sizeof(ix));
        for (int64_t x = 0; x < nx; ++x) {
          int64_t o1 = o1u, o2 = o2v;
          for (int32_t a = 0; a < s->nc; ++a) {
            o1 += st1[s->c1[a]] * ix[a];
            o2 += st2[s->c2[a]] * ix[a];
          }
          dot += d1[o1] * d2[o2];
          for (int32_t a = s->nc - 1; a >= 0; --a) {
            if (++ix[a] < ex[a]) break;
            ix[a] = 0;
          }
        }
        out[orv] += dot;
      } else {
        double gv = g[orv];
        memset(ix, 0, sizeof(ix));
        for (int64_t x = 0; x < nx; ++x) {
          int64_t o1 = o1u, o2 = o2v;
          for (int32_t a = 0; a < s->nc; ++a) {
            o1 += st1[s->c1[a]] * ix[a];
            o2 += st2[s->c2[a]] * ix[a];
          }
          if (mode == 1)
            out[o1] += scale * (gv * d2[o2]);
          else
            out[o2] += scale * (d1[o1] * gv);
          for (int32_t a = s->nc - 1; a >= 0; --a) {
            if (++ix[a] < ex[a]) break;
            ix[a] = 0;
          }
        }
      }
      for (int32_t a = s->nf2 - 1; a >= 0; --a) {
        if (++iv[a] < ev[a]) break;
        iv[a] = 0;
      }
    }
    for (int32_t a = s->nf1 - 1; a >= 0; --a) {
      if (++iu[a] < eu[a]) break;
      iu[a] = 0;
    }
  }
}

typedef struct {
  int64_t b1, b2;
} pair_t;

/* T2 blocks ordered by their contracted index tuple, for the join with T1 */
static const cset_t *g_cs;
static int cmp_t2_by_contracted(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  for (int32_t q = 0; q < g_cs->nc; ++q) {
    int32_t u = g_cs->t2.idx[x * g_cs->t2.rank + g_cs->c2[q]];
    int32_t v = g_cs->t2.idx[y * g_cs->t2.rank + g_cs->c2[q]];
    if (u != v) return u < v ? -1 : 1;
  }
  return x < y ? -1 : (x > y);
}

/* compare T1 block b1's contracted tuple with T2 block b2's */
static int cmp_contracted(const cset_t *s, int64_t b1, int64_t b2) {
  for (int32_t q = 0; q < s->nc; ++q) {
    int32_t u = s->t1.idx[b1 * s->t1.rank + s->c1[q]];
    int32_t v = s->t2.idx[b2 * s->t2.rank + s->c2[q]];
    if (u != v) return u < v ? -1 : 1;
  }
  return 0;
}

/* all kept block pairs in (b1, b2) canonical order */
static int kept_pairs(const cset_t *s, double eps, pair_t **pairs, int64_t *np, int64_t *nfilt) {
  int64_t n2 = s->t2.nblocks;
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n2 ? n2 : 1));
  if (!ord) return OR_ERR_ALLOC;
  for (int64_t b = 0; b < n2; ++b) ord[b] = b;
  g_cs = s;
  qsort(ord, (size_t)n2, sizeof(int64_t), cmp_t2_by_contracted);
  int64_t cap = 1024, n = 0, nf = 0;
  pair_t *p = (pair_t *)malloc(sizeof(pair_t) * (size_t)cap);
  if (!p) {
    free(ord);
    return OR_ERR_ALLOC;
  }
  for (int64_t b1 = 0; b1 < s->t1.nblocks; ++b1) {
    int64_t lo = 0, hi = n2;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if (cmp_contracted(s, b1, ord[mid]) > 0)
        lo = mid + 1;
      else
        hi = mid;
    }
    for (int64_t q = lo; q < n2 && cmp_contracted(s, b1, ord[q]) == 0; ++q) {
      int64_t b2 = ord[q];
      if (!pair_matches(s, b1, b2)) continue;
      if (!(s->n1[b1] * s->n2[b2] >= eps)) {
        ++nf;
        continue;
      }
      if (n == cap) {
        cap *= 2;
        pair_t *p2 = (pair_t *)realloc(p, sizeof(pair_t) * (size_t)cap);
        if (!p2) {
          free(p);
          free(ord);
          return OR_ERR_ALLOC;
        }
        p = p2;
      }
      p[n].b1 = b1;
      p[n].b2 = b2;
      ++n;
    }
  }
  free(ord);
  *pairs = p;
  *np = n;
  *nfilt = nf;
  return OR_OK;
}

static const int32_t *g_rt;
static int32_t g_rrank;
static int cmp_rtuple(const void *a, const void *b) {
  const int32_t *x = g_rt + (*(const int64_t *)a) * g_rrank;
  const int32_t *y = g_rt + (*(const int64_t *)b) * g_rrank;
  for (int32_t r = 0; r < g_rrank; ++r)
    if (x[r] != y[r]) return x[r] < y[r] ? -1 : 1;
  return 0;
}

/* R = alpha * sum over kept block pairs of the contraction of T1 and T2 over the
 * listed mode pairs + beta * R_in, with the result's modes ordered by
 * result_order (result mode r is free slot result_order[r] of (f1..., f2...)). */
int or_contract(const or_tensor *T1, const or_tensor *T2, int32_t nc, const int32_t *c1,
                const int32_t *c2, int32_t nf1, const int32_t *f1, int32_t nf2, const int32_t *f2,
                const int32_t *result_order, const or_tensor *Rin, double alpha, double beta,
                double eps, or_tresult **out) {
  *out = NULL;
  if (!(eps >= 0.0)) return OR_ERR_INVALID_ARG;
  cset_t s;
  int st = cset_make(T1, T2, nc, c1, c2, nf1, f1, nf2, f2, result_order, Rin, &s);
  if (st) return st;
  pair_t *pairs = NULL;
  int64_t np = 0, nfilt = 0;
  st = kept_pairs(&s, eps, &pairs, &np, &nfilt);
  if (st) {
    cset_free(&s);
    return st;
  }
  int32_t rr = s.rrank;
  int64_t ncand = np + (s.has_rin ? s.ri.nblocks : 0);
  int32_t *tups = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncand ? ncand : 1) * (size_t)rr);
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncand ? ncand : 1));
  or_tresult *r = (or_tresult *)calloc(1, sizeof(or_tresult));
  if (!tups || !ord || !r) {
    free(tups);
    free(ord);
    free(r);
    free(pairs);
    cset_free(&s);
    return OR_ERR_ALLOC;
  }
  for (int64_t p = 0; p < np; ++p) result_tuple(&s, pairs[p].b1, pairs[p].b2, tups + p * rr);
  for (int64_t b = 0; s.has_rin && b < s.ri.nblocks; ++b)
    memcpy(tups + (np + b) * rr, s.ri.idx + b * rr, sizeof(int32_t) * (size_t)rr);
  for (int64_t q = 0; q < ncand; ++q) ord[q] = q;
  g_rt = tups;
  g_rrank = rr;
  qsort(ord, (size_t)ncand, sizeof(int64_t), cmp_rtuple);
  /* unique result tuples, lexicographic */
  r->rank = rr;
  int64_t nsz = 0;
  for (int32_t q = 0; q < rr; ++q) {
    int32_t slot = s.ro[q];
    r->nblk[q] = slot < s.nf1 ? s.t1.nblk[s.f1[slot]] : s.t2.nblk[s.f2[slot - s.nf1]];
    nsz += r->nblk[q];
  }
  r->bsz = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsz ? nsz : 1));
  r->idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncand ? ncand : 1) * (size_t)rr);
  r->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncand ? ncand : 1));
  if (!r->bsz || !r->idx || !r->off) st = OR_ERR_ALLOC;
  tcanon_t rc;
  memset(&rc, 0, sizeof(rc));
  if (!st) {
    int64_t so = 0;
    for (int32_t q = 0; q < rr; ++q) {
      for (int32_t b = 0; b < r->nblk[q]; ++b) r->bsz[so + b] = free_slot_mode_size(&s, s.ro[q], b);
      rc.sz[q] = r->bsz + so;
      rc.nblk[q] = r->nblk[q];
      so += r->nblk[q];
    }
    rc.rank = rr;
    int64_t nu = 0;
    for (int64_t q = 0; q < ncand; ++q) {
      const int32_t *tp = tups + ord[q] * rr;
      if (nu > 0 && memcmp(r->idx + (nu - 1) * rr, tp, sizeof(int32_t) * (size_t)rr) == 0) continue;
      memcpy(r->idx + nu * rr, tp, sizeof(int32_t) * (size_t)rr);
      ++nu;
    }
    int64_t off = 0;
    for (int64_t q = 0; q < nu; ++q) {
      r->off[q] = off;
      off += tblock_len(&rc, r->idx + q * rr);
    }
    r->nblocks = nu;
    r->nelem = off;
    rc.nblocks = nu;
    rc.idx = r->idx;
    rc.off = r->off;
    r->data = (double *)calloc((size_t)(off ? off : 1), sizeof(double));
    if (!r->data) st = OR_ERR_ALLOC;
  }
  if (!st) {
    for (int64_t p = 0; p < np; ++p) {
      int32_t tp[2 * OR_MAXRANK];
      result_tuple(&s, pairs[p].b1, pairs[p].b2, tp);
      int64_t rb = tfind(&rc, tp);
      pair_kernel(&s, pairs[p].b1, pairs[p].b2, 0, NULL, r->data + r->off[rb], 1.0);
    }
    /* flops of a pair = 2 * (free elements of T1) * (free elements of T2) *
     * (contracted elements) = 2 * len(T1 block) * len(T2 block) / contracted */
    double flops = 0.0;
    for (int64_t p = 0; p < np; ++p) {
      const int32_t *t1 = s.t1.idx + pairs[p].b1 * s.t1.rank;
      double nxx = 1.0;
      for (int32_t a = 0; a < s.nc; ++a) nxx *= s.t1.sz[s.c1[a]][t1[s.c1[a]]];
      flops += 2.0 * (double)tblock_len(&s.t1, t1) *
               (double)tblock_len(&s.t2, s.t2.idx + pairs[p].b2 * s.t2.rank) / nxx;
    }
    r->flops = flops;
    for (int64_t q = 0; q < r->nblocks; ++q) {
      int64_t len = tblock_len(&rc, r->idx + q * rr);
      int64_t ib = (s.has_rin && beta != 0.0) ? tfind(&s.ri, r->idx + q * rr) : -1;
      double *c = r->data + r->off[q];
      for (int64_t e = 0; e < len; ++e) {
        double v = alpha * c[e];
        if (ib >= 0) v += beta * s.ri.data[s.ri.off[ib] + e];
        c[e] = v;
      }
    }
    r->npairs = np;
    r->nfiltered = nfilt;
  }
  free(tups);
  free(ord);
  free(pairs);
  cset_free(&s);
  if (st) {
    or_tresult_free(r);
    return st;
  }
  *out = r;
  return OR_OK;
}

/* Adjoint of or_contract with the filter decisions held fixed: given dR packed in
 * the canonical result order that or_contract returns,
 *   dT1[u,x] = alpha * sum over kept pairs of sum_v dR[u,v] T2[x,v]  (pattern of T1),
 *   dT2[x,v] = alpha * sum over kept pairs of sum_u T1[u,x] dR[u,v]  (pattern of T2),
 *   dR_in    = beta * dR                                              (pattern of R_in),
 * each in the canonical packing of its own tensor. */
int or_contract_adjoint(const or_tensor *T1, const or_tensor *T2, int32_t nc, const int32_t *c1,
                        const int32_t *c2, int32_t nf1, const int32_t *f1, int32_t nf2,
                        const int32_t *f2, const int32_t *result_order, const or_tensor *Rin,
                        double alpha, double beta, double eps, const double *dR, double *dT1,
                        double *dT2, double *dRin) {
  or_tresult *res = NULL;
  int st = or_contract(T1, T2, nc, c1, c2, nf1, f1, nf2, f2, result_order, Rin, alpha, beta, eps,
                       &res);
  if (st) return st;
  cset_t s;
  st = cset_make(T1, T2, nc, c1, c2, nf1, f1, nf2, f2, result_order, Rin, &s);
  if (st) {
    or_tresult_free(res);
    return st;
  }
  pair_t *pairs = NULL;
  int64_t np = 0, nfilt = 0;
  st = kept_pairs(&s, eps, &pairs, &np, &nfilt);
  if (st) {
    cset_free(&s);
    or_tresult_free(res);
    return st;
  }
  tcanon_t rc;
  memset(&rc, 0, sizeof(rc));
  rc.rank = res->rank;
  {
    int64_t so = 0;
    for (int32_t q = 0; q < res->rank; ++q) {
      rc.nblk[q] = res->nblk[q];
      rc.sz[q] = res->bsz + so;
      so += res->nblk[q];
    }
  }
  rc.nblocks = res->nblocks;
  rc.idx = res->idx;
  rc.off = res->off;
  memset(dT1, 0, sizeof(double) * (size_t)s.t1.nelem);
  memset(dT2, 0, sizeof(double) * (size_t)s.t2.nelem);
  for (int64_t p = 0; p < np; ++p) {
    int32_t tp[2 * OR_MAXRANK];
    result_tuple(&s, pairs[p].b1, pairs[p].b2, tp);
    const double *g = dR + res->off[tfind(&rc, tp)];
    pair_kernel(&s, pairs[p].b1, pairs[p].b2, 1, g, dT1 + s.t1.off[pairs[p].b1], alpha);
    pair_kernel(&s, pairs[p].b1, pairs[p].b2, 2, g, dT2 + s.t2.off[pairs[p].b2], alpha);
  }
  if (s.has_rin && dRin) {
    for (int64_t b = 0; b < s.ri.nblocks; ++b) {
      int64_t q = tfind(&rc, s.ri.idx + b * s.ri.rank);
      int64_t len = tblock_len(&s.ri, s.ri.idx + b * s.ri.rank);
      for (int64_t e = 0; e < len; ++e) dRin[s.ri.off[b] + e] = beta * dR[res->off[q] + e];
    }
  }
  free(pairs);
  cset_free(&s);
  or_tresult_free(res);
  return OR_OK;
}

/* Values of selected result blocks only (tuples req[nreq * rank] in the result's mode
 * order), from the same definition as or_contract: alpha * the sum over the kept block
 * pairs that land on each requested block + beta * R_in.  out is packed in request
 * order, each block row-major; present[e] = 0 for a block outside the result pattern
 * (its values come back as zeros). */
int or_contract_sample(const or_tensor *T1, const or_tensor *T2, int32_t nc, const int32_t *c1,
                       const int32_t *c2, int32_t nf1, const int32_t *f1, int32_t nf2,
                       const int32_t *f2, const int32_t *result_order, const or_tensor *Rin,
                       double alpha, double beta, double eps, int64_t nreq, const int32_t *req,
                       double *out, int8_t *present) {
  if (!(eps >= 0.0)) return OR_ERR_INVALID_ARG;
  cset_t s;
  int st = cset_make(T1, T2, nc, c1, c2, nf1, f1, nf2, f2, result_order, Rin, &s);
  if (st) return st;
  pair_t *pairs = NULL;
  int64_t np = 0, nfilt = 0;
  st = kept_pairs(&s, eps, &pairs, &np, &nfilt);
  if (st) {
    cset_free(&s);
    return st;
  }
  int32_t rr = s.rrank;
  /* block sizes of the result modes, and the requested blocks in canonical form */
  int32_t rnblk[2 * OR_MAXRANK];
  tcanon_t rq;
  memset(&rq, 0, sizeof(rq));
  rq.rank = rr;
  int32_t *rsz_all = NULL;
  {
    int64_t tot = 0;
    for (int32_t q = 0; q < rr; ++q) {
      int32_t slot = s.ro[q];
      rnblk[q] = slot < s.nf1 ? s.t1.nblk[s.f1[slot]] : s.t2.nblk[s.f2[slot - s.nf1]];
      tot += rnblk[q];
    }
    rsz_all = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot ? tot : 1));
    if (!rsz_all) {
      free(pairs);
      cset_free(&s);
      return OR_ERR_ALLOC;
    }
    int64_t so = 0;
    for (int32_t q = 0; q < rr; ++q) {
      for (int32_t b = 0; b < rnblk[q]; ++b) rsz_all[so + b] = free_slot_mode_size(&s, s.ro[q], b);
      rq.sz[q] = rsz_all + so;
      rq.nblk[q] = rnblk[q];
      so += rnblk[q];
    }
  }
  int64_t *roff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nreq ? nreq : 1));
  if (!roff) st = OR_ERR_ALLOC;
  int64_t total = 0;
  for (int64_t e = 0; !st && e < nreq; ++e) {
    for (int32_t q = 0; q < rr; ++q)
      if (req[e * rr + q] < 0 || req[e * rr + q] >= rnblk[q]) st = OR_ERR_OUT_OF_RANGE;
    if (st) break;
    roff[e] = total;
    total += tblock_len(&rq, req + e * rr);
    present[e] = 0;
  }
  if (!st) {
    for (int64_t x = 0; x < total; ++x) out[x] = 0.0;
    for (int64_t p = 0; p < np; ++p) {
      int32_t tp[2 * OR_MAXRANK];
      result_tuple(&s, pairs[p].b1, pairs[p].b2, tp);
      for (int64_t e = 0; e < nreq; ++e) {
        if (memcmp(tp, req + e * rr, sizeof(int32_t) * (size_t)rr) != 0) continue;
        pair_kernel(&s, pairs[p].b1, pairs[p].b2, 0, NULL, out + roff[e], 1.0);
        present[e] = 1;
      }
    }
    for (int64_t e = 0; e < nreq; ++e) {
      int64_t ib = s.has_rin ? tfind(&s.ri, req + e * rr) : -1;
      if (ib >= 0) present[e] = 1;
      int64_t len = tblock_len(&rq, req + e * rr);
      for (int64_t x = 0; x < len; ++x) {
        double v = alpha * out[roff[e] + x];
        if (ib >= 0 && beta != 0.0) v += beta * s.ri.data[s.ri.off[ib] + x];
        out[roff[e] + x] = v;
      }
    }
  }
  free(roff);
  free(rsz_all);
  free(pairs);
  cset_free(&s);
  return st;
}
