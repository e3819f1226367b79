/*
 * Seeded synthetic inputs for the exponential-shift low-diameter
 * decomposition (Miller, Peng, Xu, "Parallel Graph Decompositions Using
 * Random Shifts", 2013).
 *
 * This file holds none of the decomposition's arithmetic.  It produces the
 * two inputs the method consumes:
 *   - an undirected, unweighted graph as a symmetric int32 CSR (Definition 1.1
 *     of the paper fixes the input class; the generators themselves are not in
 *     the paper): 2D / 3D lattice grids, R-MAT, random geometric graphs;
 *   - the per-vertex shifts delta_u ~ Exp(beta) of Algorithm 2 step 1, drawn in
 *     FP64 from a counter-based generator so that every consumer sees the same
 *     array.
 *
 * Random numbers come from Philox4x32-10, written from its published
 * definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): a 4x32-bit counter, a 2x32-bit key, ten rounds of two
 * 32x32->64 multiplies with the key bumped by two Weyl constants between
 * rounds.
 *
 * Counter layouts (fixed here, recorded by every consumer):
 *   shifts : counter = (u_lo, u_hi, 0, 0), key = (seed_lo, seed_hi);
 *            w = ((x0 << 32) | x1) >> 11  (53 bits),  U = (w + 1) * 2^-53 in (0,1],
 *            delta_u = -log(U) / beta.
 *   R-MAT  : counter = (i_lo, i_hi, j, 1) gives the 32-bit draws of levels
 *            4j..4j+3 of edge i.
 *   RGG    : counter = (i_lo, i_hi, 0, 2) gives point i: x from (x0,x1),
 *            y from (x2,x3), each 53 bits scaled by 2^-53 into [0,1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void ldd_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += PHILOX_W0;
      k[1] += PHILOX_W1;
    }
    philox_round(c, k);
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

/* Raw words for counters (i_lo, i_hi, w2, w3), i in [first, first+count). */
void ldd_philox_stream(uint64_t seed, uint64_t first, int64_t count, uint32_t w2, uint32_t w3,
                       uint32_t* out /* [count*4] */) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    uint64_t c = first + (uint64_t)i;
    uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), w2, w3};
    ldd_philox4x32_10(ctr, key, out + 4 * i);
  }
}

/* ------------------------------------------------------------------ */
/* Shifts delta_u ~ Exp(beta)                                          */
/* ------------------------------------------------------------------ */
/* Uniforms U_u in (0,1]: exposed separately so tests can check the map. */
void ldd_gen_uniforms(int64_t n, uint64_t seed, double* out) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int64_t u = 0; u < n; ++u) {
    uint32_t ctr[4] = {(uint32_t)u, (uint32_t)((uint64_t)u >> 32), 0u, 0u}, x[4];
    ldd_philox4x32_10(ctr, key, x);
    uint64_t w = (((uint64_t)x[0] << 32) | x[1]) >> 11;
    out[u] = (double)(w + 1) * 0x1.0p-53;
  }
}

/* Inverse-CDF draw of the exponential distribution (paper, Section 2:
 * F(x) = 1 - exp(-beta x); with U uniform on (0,1], -ln(U)/beta ~ Exp(beta)). */
void ldd_gen_shifts(int64_t n, double beta, uint64_t seed, double* out) {
  ldd_gen_uniforms(n, seed, out);
#pragma omp parallel for schedule(static)
  for (int64_t u = 0; u < n; ++u) {
    double d = -log(out[u]) / beta;
    out[u] = (d == 0.0) ? 0.0 : d; /* U == 1 gives -0.0; store +0.0 */
  }
}

/* ------------------------------------------------------------------ */
/* Lattice grids (ids row-major, neighbour lists ascending)            */
/* ------------------------------------------------------------------ */
int64_t ldd_grid2d_nnz(int64_t nx, int64_t ny) {
  return 2 * ((nx - 1) * ny + nx * (ny - 1));
}

void ldd_gen_grid2d(int64_t nx, int64_t ny, int32_t* row_ptr, int32_t* col) {
  int64_t n = nx * ny;
  /* degrees -> prefix sums (row-major order keeps it sequential) */
  row_ptr[0] = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t x = v % nx, y = v / nx;
    int d = (y > 0) + (x > 0) + (x + 1 < nx) + (y + 1 < ny);
    row_ptr[v + 1] = row_ptr[v] + d;
  }
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    int64_t x = v % nx, y = v / nx;
    int32_t* p = col + row_ptr[v];
    if (y > 0) *p++ = (int32_t)(v - nx);
    if (x > 0) *p++ = (int32_t)(v - 1);
    if (x + 1 < nx) *p++ = (int32_t)(v + 1);
    if (y + 1 < ny) *p++ = (int32_t)(v + nx);
  }
}

int64_t ldd_grid3d_nnz(int64_t nx, int64_t ny, int64_t nz) {
  return 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1));
}

void ldd_gen_grid3d(int64_t nx, int64_t ny, int64_t nz, int32_t* row_ptr, int32_t* col) {
  int64_t n = nx * ny * nz, plane = nx * ny;
  row_ptr[0] = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t x = v % nx, y = (v / nx) % ny, z = v / plane;
    int d = (z > 0) + (y > 0) + (x > 0) + (x + 1 < nx) + (y + 1 < ny) + (z + 1 < nz);
    row_ptr[v + 1] = row_ptr[v] + d;
  }
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    int64_t x = v % nx, y = (v / nx) % ny, z = v / plane;
    int32_t* p = col + row_ptr[v];
    if (z > 0) *p++ = (int32_t)(v - plane);
    if (y > 0) *p++ = (int32_t)(v - nx);
    if (x > 0) *p++ = (int32_t)(v - 1);
    if (x + 1 < nx) *p++ = (int32_t)(v + 1);
    if (y + 1 < ny) *p++ = (int32_t)(v + nx);
    if (z + 1 < nz) *p++ = (int32_t)(v + plane);
  }
}

/* ------------------------------------------------------------------ */
/* Edge list -> symmetric CSR without self-loops or duplicate arcs      */
/* ------------------------------------------------------------------ */
static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void sort_row(int32_t* p, int64_t len) {
  if (len < 24) {
    for (int64_t i = 1; i < len; ++i) {
      int32_t t = p[i];
      int64_t j = i - 1;
      while (j >= 0 && p[j] > t) {
        p[j + 1] = p[j];
        --j;
      }
      p[j + 1] = t;
    }
  } else {
    qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
  }
}

/* Builds the CSR into malloc'd buffers; returns nnz, or -1 on failure. */
static int64_t edges_to_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                            int32_t** row_ptr_out, int32_t** col_out) {
  int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!start) return -1;
  for (int64_t i = 0; i < m; ++i) {
    if (src[i] == dst[i]) continue;
    start[src[i] + 1]++;
    start[dst[i] + 1]++;
  }
  for (int64_t v = 0; v < n; ++v) start[v + 1] += start[v];
  int64_t total = start[n];
  int32_t* tmp = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  int64_t* fill = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!tmp || !fill) {
    free(start);
    free(tmp);
    free(fill);
    return -1;
  }
  memcpy(fill, start, (size_t)n * sizeof(int64_t));
  for (int64_t i = 0; i < m; ++i) {
    int32_t u = src[i], v = dst[i];
    if (u == v) continue;
    tmp[fill[u]++] = v;
    tmp[fill[v]++] = u;
  }
  free(fill);
  int32_t* newdeg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!newdeg) {
    free(start);
    free(tmp);
    return -1;
  }
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v) {
    int32_t* p = tmp + start[v];
    int64_t len = start[v + 1] - start[v];
    sort_row(p, len);
    int64_t k = 0;
    for (int64_t i = 0; i < len; ++i)
      if (k == 0 || p[i] != p[k - 1]) p[k++] = p[i];
    newdeg[v] = (int32_t)k;
  }
  int32_t* row_ptr = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  if (!row_ptr) {
    free(start);
    free(tmp);
    free(newdeg);
    return -1;
  }
  int64_t acc = 0;
  row_ptr[0] = 0;
  for (int64_t v = 0; v < n; ++v) {
    acc += newdeg[v];
    if (acc > INT32_MAX) {
      free(start);
      free(tmp);
      free(newdeg);
      free(row_ptr);
      return -1;
    }
    row_ptr[v + 1] = (int32_t)acc;
  }
  int32_t* col = (int32_t*)malloc((size_t)(acc > 0 ? acc : 1) * sizeof(int32_t));
  if (!col) {
    free(start);
    free(tmp);
    free(newdeg);
    free(row_ptr);
    return -1;
  }
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v)
    memcpy(col + row_ptr[v], tmp + start[v], (size_t)newdeg[v] * sizeof(int32_t));
  free(start);
  free(tmp);
  free(newdeg);
  *row_ptr_out = row_ptr;
  *col_out = col;
  return acc;
}

void ldd_gen_free(void* p) { free(p); }

/* ------------------------------------------------------------------ */
/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): each of the m = ef * 2^scale
 * edges picks one quadrant per level with probabilities (a, b, c, d);
 * a = (row 0, col 0), b = (0, 1), c = (1, 0), d = (1, 1), most significant
 * level first.  No noise, no relabelling.  Symmetrised, self-loops and
 * duplicate arcs removed.                                              */
/* ------------------------------------------------------------------ */
int64_t ldd_gen_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
                     int32_t** row_ptr_out, int32_t** col_out) {
  if (scale < 1 || scale > 30) return -1;
  int64_t n = (int64_t)1 << scale;
  int64_t m = edge_factor * n;
  const uint64_t ta = (uint64_t)(a * 4294967296.0);
  const uint64_t tab = (uint64_t)((a + b) * 4294967296.0);
  const uint64_t tabc = (uint64_t)((a + b + c) * 4294967296.0);
  int32_t* src = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  if (!src || !dst) {
    free(src);
    free(dst);
    return -1;
  }
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const int nblk = (scale + 3) / 4;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    uint32_t u = 0, v = 0;
    for (int j = 0; j < nblk; ++j) {
      uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)j, 1u}, x[4];
      ldd_philox4x32_10(ctr, key, x);
      for (int t = 0; t < 4; ++t) {
        int l = 4 * j + t;
        if (l >= scale) break;
        uint32_t bit = 1u << (scale - 1 - l);
        uint64_t w = x[t];
        if (w < ta) {
        } else if (w < tab) {
          v |= bit;
        } else if (w < tabc) {
          u |= bit;
        } else {
          u |= bit;
          v |= bit;
        }
      }
    }
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
  int64_t nnz = edges_to_csr(n, m, src, dst, row_ptr_out, col_out);
  free(src);
  free(dst);
  return nnz;
}

/* ------------------------------------------------------------------ */
/* Random geometric graph in the unit square: n points uniform in [0,1)^2,
 * an edge between two points at Euclidean distance < radius.  Cell-grid
 * bucketing with cell side >= radius.                                  */
/* ------------------------------------------------------------------ */
int64_t ldd_gen_rgg(int64_t n, double radius, uint64_t seed, int32_t** row_ptr_out,
                    int32_t** col_out) {
  if (n < 1 || radius <= 0.0) return -1;
  double* px = (double*)malloc((size_t)n * sizeof(double));
  double* py = (double*)malloc((size_t)n * sizeof(double));
  if (!px || !py) {
    free(px);
    free(py);
    return -1;
  }
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 2u}, x[4];
    ldd_philox4x32_10(ctr, key, x);
    px[i] = (double)((((uint64_t)x[0] << 32) | x[1]) >> 11) * 0x1.0p-53;
    py[i] = (double)((((uint64_t)x[2] << 32) | x[3]) >> 11) * 0x1.0p-53;
  }
  int64_t g = (int64_t)floor(1.0 / radius);
  if (g < 1) g = 1;
  if (g > 65536) g = 65536;
  int64_t ncell = g * g;
  int64_t* cstart = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  int32_t* cell_of = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* members = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!cstart || !cell_of || !members) {
    free(px);
    free(py);
    free(cstart);
    free(cell_of);
    free(members);
    return -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = (int64_t)(px[i] * g), cy = (int64_t)(py[i] * g);
    if (cx >= g) cx = g - 1;
    if (cy >= g) cy = g - 1;
    cell_of[i] = (int32_t)(cy * g + cx);
    cstart[cell_of[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  {
    int64_t* fill = (int64_t*)malloc((size_t)ncell * sizeof(int64_t));
    if (!fill) {
      free(px);
      free(py);
      free(cstart);
      free(cell_of);
      free(members);
      return -1;
    }
    memcpy(fill, cstart, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) members[fill[cell_of[i]]++] = (int32_t)i;
    free(fill);
  }
  const double r2 = radius * radius;
  /* count, then fill, rows directly (each pair seen from both ends) */
  int32_t* deg = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  if (!deg) {
    free(px);
    free(py);
    free(cstart);
    free(cell_of);
    free(members);
    return -1;
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = cell_of[i] % g, cy = cell_of[i] / g;
    int32_t d = 0;
    for (int64_t yy = cy - 1; yy <= cy + 1; ++yy)
      for (int64_t xx = cx - 1; xx <= cx + 1; ++xx) {
        if (xx < 0 || yy < 0 || xx >= g || yy >= g) continue;
        int64_t c = yy * g + xx;
        for (int64_t k = cstart[c]; k < cstart[c + 1]; ++k) {
          int32_t j = members[k];
          if (j == i) continue;
          double dx = px[i] - px[j], dy = py[i] - py[j];
          if (dx * dx + dy * dy < r2) ++d;
        }
      }
    deg[i] = d;
  }
  int32_t* row_ptr = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int64_t acc = 0;
  if (row_ptr) {
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
      acc += deg[i];
      if (acc > INT32_MAX) break;
      row_ptr[i + 1] = (int32_t)acc;
    }
  }
  int32_t* col = (row_ptr && acc <= INT32_MAX)
                     ? (int32_t*)malloc((size_t)(acc > 0 ? acc : 1) * sizeof(int32_t))
                     : NULL;
  if (!col) {
    free(px);
    free(py);
    free(cstart);
    free(cell_of);
    free(members);
    free(deg);
    free(row_ptr);
    return -1;
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = cell_of[i] % g, cy = cell_of[i] / g;
    int32_t* p = col + row_ptr[i];
    int64_t len = 0;
    for (int64_t yy = cy - 1; yy <= cy + 1; ++yy)
      for (int64_t xx = cx - 1; xx <= cx + 1; ++xx) {
        if (xx < 0 || yy < 0 || xx >= g || yy >= g) continue;
        int64_t c = yy * g + xx;
        for (int64_t k = cstart[c]; k < cstart[c + 1]; ++k) {
          int32_t j = members[k];
          if (j == i) continue;
          double dx = px[i] - px[j], dy = py[i] - py[j];
          if (dx * dx + dy * dy < r2) p[len++] = j;
        }
      }
    sort_row(p, len);
  }
  free(px);
  free(py);
  free(cstart);
  free(cell_of);
  free(members);
  free(deg);
  *row_ptr_out = row_ptr;
  *col_out = col;
  return acc;
}
