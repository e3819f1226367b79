/*
 * ORACLE -- test infrastructure only.  Plain, single-threaded CPU reference
 * for the exponential-shift low-diameter decomposition of Miller, Peng and Xu,
 * "Parallel Graph Decompositions Using Random Shifts" (2013).  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may
 * load this.  It shares no code with the CUDA library.
 *
 * What it computes (Algorithm 2, Eq. (1)): every vertex v is assigned to the
 * vertex u minimising the shifted distance dist(u, v) - delta_u, ties broken
 * towards the smaller vertex id ("lexicographically", Algorithm 2 step 2; the
 * tie case is also the second case of the proof of Lemma 3.1).  Output:
 * center[v] = that u, dist[v] = dist(u, v).
 *
 * How: Section 4's first observation -- a super source s joined to every u
 * with length -delta_u -- turns the all-pairs argmin into one single-source
 * shortest-path problem; the piece of v is the first vertex after s on its
 * shortest path.  Here that is a multi-source Dijkstra in which u starts with
 * label -delta_u (no delta_max offset is needed: a priority queue takes
 * negative start labels directly).  A label is carried as the exact triple
 *     (I, f, c) = (dist - floor(delta_c), delta_c - floor(delta_c), c)
 * with value dist - delta_c = I - f.  Section 4 notes that fractional parts
 * only matter when integer parts tie; since f lies in [0, 1),
 *     I1 - f1 < I2 - f2   <=>   I1 < I2, or I1 == I2 and f1 > f2,
 * and the remaining exact ties go to the smaller c.  floor() and the
 * subtraction delta - floor(delta) are exact in FP64 (Sterbenz), so every
 * comparison is exact.  Each edge has length 1, so a relaxation v -> w
 * offers w the label (I_v + 1, f_v, c_v).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
  int64_t* I;   /* integer part of the label: dist - floor(delta_center) */
  double* F;    /* fractional part of delta_center */
  int32_t* C;   /* center id */
  int32_t* D;   /* hop distance to the center */
  int32_t* heap;
  int64_t* pos; /* heap position of a vertex, -1 once removed */
  int64_t size;
} state_t;

/* (I1,F1,C1) < (I2,F2,C2) in the exact order of dist - delta, then id. */
static inline int label_less(int64_t I1, double F1, int32_t C1, int64_t I2, double F2,
                             int32_t C2) {
  if (I1 != I2) return I1 < I2;
  if (F1 != F2) return F1 > F2;
  return C1 < C2;
}

static inline int vless(const state_t* s, int32_t a, int32_t b) {
  return label_less(s->I[a], s->F[a], s->C[a], s->I[b], s->F[b], s->C[b]);
}

static void sift_up(state_t* s, int64_t i) {
  int32_t v = s->heap[i];
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!vless(s, v, s->heap[p])) break;
    s->heap[i] = s->heap[p];
    s->pos[s->heap[i]] = i;
    i = p;
  }
  s->heap[i] = v;
  s->pos[v] = i;
}

static void sift_down(state_t* s, int64_t i) {
  int32_t v = s->heap[i];
  for (;;) {
    int64_t l = 2 * i + 1;
    if (l >= s->size) break;
    int64_t b = l;
    if (l + 1 < s->size && vless(s, s->heap[l + 1], s->heap[l])) b = l + 1;
    if (!vless(s, s->heap[b], v)) break;
    s->heap[i] = s->heap[b];
    s->pos[s->heap[i]] = i;
    i = b;
  }
  s->heap[i] = v;
  s->pos[v] = i;
}

/* Returns 0 on success, -1 for a shift that is NaN or negative, -2 on
 * allocation failure. */
int oracle_ldd(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* delta,
               int32_t* center, int32_t* dist) {
  for (int64_t u = 0; u < n; ++u)
    if (!(delta[u] >= 0.0) || isinf(delta[u])) return -1;
  if (n == 0) return 0;
  state_t s;
  s.I = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  s.F = (double*)malloc((size_t)n * sizeof(double));
  s.C = center;
  s.D = dist;
  s.heap = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  s.pos = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  double* fr = (double*)malloc((size_t)n * sizeof(double));
  int64_t* fl = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!s.I || !s.F || !s.heap || !s.pos || !fr || !fl) {
    free(s.I);
    free(s.F);
    free(s.heap);
    free(s.pos);
    free(fr);
    free(fl);
    return -2;
  }
  /* Every u starts as its own candidate center: label -delta_u. */
  for (int64_t u = 0; u < n; ++u) {
    double a = floor(delta[u]);
    fl[u] = (int64_t)a;
    fr[u] = delta[u] - a;
    s.I[u] = -fl[u];
    s.F[u] = fr[u];
    s.C[u] = (int32_t)u;
    s.D[u] = 0;
    s.heap[u] = (int32_t)u;
    s.pos[u] = u;
  }
  s.size = n;
  for (int64_t i = n / 2 - 1; i >= 0; --i) sift_down(&s, i);

  while (s.size > 0) {
    int32_t v = s.heap[0];
    s.pos[v] = -1;
    s.size--;
    if (s.size > 0) {
      s.heap[0] = s.heap[s.size];
      s.pos[s.heap[0]] = 0;
      sift_down(&s, 0);
    }
    /* v's label is final; offer (I_v + 1, f_v, c_v) to every neighbour. */
    const int64_t I1 = s.I[v] + 1;
    const double F1 = s.F[v];
    const int32_t C1 = s.C[v];
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int32_t w = col[e];
      if (s.pos[w] < 0) continue; /* already final */
      if (label_less(I1, F1, C1, s.I[w], s.F[w], s.C[w])) {
        s.I[w] = I1;
        s.F[w] = F1;
        s.C[w] = C1;
        s.D[w] = s.D[v] + 1;
        sift_up(&s, s.pos[w]);
      }
    }
  }
  free(s.I);
  free(s.F);
  free(s.heap);
  free(s.pos);
  free(fr);
  free(fl);
  return 0;
}

/* Number of undirected edges whose endpoints lie in different pieces
 * (Definition 1.1, second condition): arcs (v, w) with v < w and
 * center[v] != center[w], so each edge of a symmetric CSR counts once. */
int64_t oracle_cut_edges(int64_t n, const int32_t* row_ptr, const int32_t* col,
                         const int32_t* center) {
  int64_t cut = 0;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int32_t w = col[e];
      if (v < w && center[v] != center[w]) ++cut;
    }
  return cut;
}

/*
 * Optimality certificate for a claimed assignment (center, dist), checked in
 * O(n + m) with the same exact label order as above.  A labelling of the
 * super-source shortest-path problem of Section 4 is the optimum iff
 *   (a) it is achieved: every center c has center[c] = c, dist[c] = 0, and
 *       every other v has a neighbour w in the same piece with
 *       dist[w] = dist[v] - 1 (the predecessor of Lemma 3.1), so the label is
 *       the length of a real path from its center;
 *   (b) it cannot be improved: no vertex's own start label -delta_v and no
 *       neighbour's label + 1 is smaller than it.
 * (a) bounds the label from below by the optimum, (b) from above.  Returns 0
 * when the certificate holds, otherwise a positive code (1 = bad center,
 * 2 = center not its own, 3 = no predecessor, 4 = improvable by own start,
 * 5 = improvable by a neighbour) and writes the offending vertex to *bad.
 */
int oracle_certify(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* delta,
                   const int32_t* center, const int32_t* dist, int64_t* bad) {
  for (int64_t v = 0; v < n; ++v) {
    int32_t c = center[v];
    if (c < 0 || c >= n || dist[v] < 0) {
      *bad = v;
      return 1;
    }
    if (center[c] != c || dist[c] != 0) {
      *bad = v;
      return 2;
    }
    if (c != v) {
      int ok = 0;
      for (int64_t e = row_ptr[v]; e < row_ptr[v + 1] && !ok; ++e) {
        int32_t w = col[e];
        ok = (center[w] == c && dist[w] == dist[v] - 1);
      }
      if (!ok) {
        *bad = v;
        return 3;
      }
    }
  }
  for (int64_t v = 0; v < n; ++v) {
    int32_t c = center[v];
    double ac = floor(delta[c]);
    int64_t Iv = (int64_t)dist[v] - (int64_t)ac;
    double Fv = delta[c] - ac;
    double av = floor(delta[v]);
    if (label_less(-(int64_t)av, delta[v] - av, (int32_t)v, Iv, Fv, c)) {
      *bad = v;
      return 4;
    }
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      int32_t w = col[e];
      int32_t cw = center[w];
      double aw = floor(delta[cw]);
      int64_t Iw = (int64_t)dist[w] - (int64_t)aw;
      if (label_less(Iw + 1, delta[cw] - aw, cw, Iv, Fv, c)) {
        *bad = v;
        return 5;
      }
    }
  }
  return 0;
}
