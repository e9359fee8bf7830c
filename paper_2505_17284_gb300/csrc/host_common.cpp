// Instance construction for the S_N step: validation, mesh metadata (Sec. 4.2),
// time step (Sec. 4.3), device buffers, TMA tensor maps and work items.
#include "host_common.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <unordered_map>

namespace rtk {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}
void clear_error() { g_last_error.clear(); }
const char* last_error_cstr() { return g_last_error.c_str(); }

rt_status DeviceArena::get(size_t n, void** out) {
  *out = nullptr;
  if (n == 0) n = 256;
  n = (n + 255) / 256 * 256;
  void* p = nullptr;
  if (alloc_fn) {
    p = alloc_fn(n, ctx);
    if (!p) {
      set_error("allocator returned NULL for %zu bytes", n);
      return RT_ENOMEM;
    }
  } else {
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      set_error("cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
    }
  }
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0) {
    set_error("allocator returned a pointer that is not 16-byte aligned");
    if (free_fn) free_fn(p, ctx); else cudaFree(p);
    return RT_EINVAL;
  }
  owned.push_back(p);
  bytes += (int64_t)n;
  *out = p;
  return RT_OK;
}

void DeviceArena::release(void* p) {
  auto it = std::find(owned.begin(), owned.end(), p);
  if (it == owned.end()) return;
  owned.erase(it);
  if (free_fn) free_fn(p, ctx); else cudaFree(p);
}

void DeviceArena::free_all() {
  for (void* p : owned) {
    if (free_fn) free_fn(p, ctx); else cudaFree(p);
  }
  owned.clear();
}

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return n;
}

// ---------------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

static rt_status encode_psi_map(CUtensorMap* map, void* base, int storage, int Mpad, int nx, int ny, int box_k,
                                int box_x) {
  auto enc = get_encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return RT_ECUDA;
  }
  const size_t es = storage == RT_BF16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)Mpad, (cuuint64_t)nx, (cuuint64_t)ny};
  cuuint64_t strides[2] = {(cuuint64_t)Mpad * es, (cuuint64_t)nx * Mpad * es};
  cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_x, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(map, storage == RT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                   base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for dims {%d,%d,%d} box_x %d", (int)r, Mpad, nx, ny, box_x);
    return RT_ECUDA;
  }
  return RT_OK;
}

// ---------------------------------------------------------------- validation
static bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

static rt_status validate_common(const rt_materials* mat, const rt_quadrature* quad, const rt_boundary* bc,
                                 int order, int integrator, int storage, double t_end, int64_t n_cells) {
  if (!mat || !quad || !bc) { set_error("materials, quadrature and boundary are required"); return RT_EINVAL; }
  if (order != 1 && order != 2) { set_error("order must be 1 or 2 (got %d)", order); return RT_EINVAL; }
  if (integrator != RT_EULER && integrator != RT_HEUN) { set_error("integrator must be RT_EULER or RT_HEUN"); return RT_EINVAL; }
  if (storage != RT_FP32 && storage != RT_BF16) { set_error("storage must be RT_FP32 or RT_BF16"); return RT_EINVAL; }
  if (!(t_end > 0.0) || !std::isfinite(t_end)) { set_error("t_end must be positive and finite"); return RT_EINVAL; }
  if (mat->n_mat < 1 || mat->n_mat > RT_MAX_MATERIALS) { set_error("n_mat must be in 1..%d", RT_MAX_MATERIALS); return RT_EINVAL; }
  if (mat->n_regions < 1 || mat->n_regions > RT_MAX_REGIONS) { set_error("n_regions must be in 1..%d", RT_MAX_REGIONS); return RT_EINVAL; }
  if (!mat->sigma_a || !mat->sigma_s || !mat->Q || !mat->cell_mat || !mat->cell_region) {
    set_error("material arrays must not be NULL"); return RT_EINVAL;
  }
  for (int m = 0; m < mat->n_mat; ++m) {
    if (!finite_nonneg(mat->sigma_a[m]) || !finite_nonneg(mat->sigma_s[m]) || !std::isfinite(mat->Q[m])) {
      set_error("material %d: sigma_a, sigma_s must be finite and >= 0, Q finite", m); return RT_EINVAL;
    }
  }
  for (int64_t i = 0; i < n_cells; ++i) {
    if (mat->cell_mat[i] < 0 || mat->cell_mat[i] >= mat->n_mat) { set_error("cell %lld: material id %d out of range", (long long)i, mat->cell_mat[i]); return RT_EINVAL; }
    if (mat->cell_region[i] < 0 || mat->cell_region[i] >= mat->n_regions) { set_error("cell %lld: region id %d out of range", (long long)i, mat->cell_region[i]); return RT_EINVAL; }
  }
  if (quad->M < 1 || quad->M > 65536 || !quad->xi || !quad->eta || !quad->w) { set_error("quadrature: need 1 <= M <= 65536 and non-NULL arrays"); return RT_EINVAL; }
  for (int64_t k = 0; k < quad->M; ++k) {
    const double x = quad->xi[k], y = quad->eta[k], w = quad->w[k];
    if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(w) || x * x + y * y > 1.0 + 1e-12 || w < 0.0) {
      set_error("ordinate %lld: need finite xi, eta with xi^2 + eta^2 <= 1 and w >= 0", (long long)k); return RT_EINVAL;
    }
  }
  for (int s = 0; s < 4; ++s) {
    const int k = bc->side_kind[s];
    if (k != RT_BC_VACUUM && k != RT_BC_INFLOW && k != RT_BC_PERIODIC) { set_error("side %d: unknown boundary kind %d", s, k); return RT_EINVAL; }
    if (k == RT_BC_INFLOW && !std::isfinite(bc->inflow[s])) { set_error("side %d: inflow must be finite", s); return RT_EINVAL; }
  }
  for (int a = 0; a < 2; ++a)
    if ((bc->side_kind[2 * a] == RT_BC_PERIODIC) != (bc->side_kind[2 * a + 1] == RT_BC_PERIODIC)) {
      set_error("periodic sides come in pairs (x-/x+ or y-/y+)"); return RT_EINVAL;
    }
  return RT_OK;
}

static int64_t steps_for(double t_end, double dt_target) {
  const double r = t_end / dt_target - 1e-9;
  int64_t n = (int64_t)std::ceil(r);
  return n < 1 ? 1 : n;
}

// ---------------------------------------------------------------- triangles
struct TriMeta {
  std::vector<int4> nbr;
  std::vector<float4> geo;
  std::vector<float4> geo2;   // second order: centroid-to-midpoint and centroid-to-neighbour vectors
  std::vector<double> area;
  double min_2a_over_p = 0;
};

static rt_status triangle_metadata(const rt_mesh* m, const int32_t* cell_mat, const int32_t* cell_reg, TriMeta& out) {
  const int64_t nv = m->n_vert, nt = m->n_tri;
  const double* V = m->vxy;
  const int32_t* T = m->tri;
  if (nv < 3 || nt < 1 || !V || !T) { set_error("triangle mesh: need n_vert >= 3, n_tri >= 1 and arrays"); return RT_EINVAL; }
  if (nt > (int64_t)0x7fffffff / 2) { set_error("triangle mesh too large"); return RT_EINVAL; }
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  for (int64_t v = 0; v < nv; ++v) {
    const double x = V[2 * v], y = V[2 * v + 1];
    if (!std::isfinite(x) || !std::isfinite(y)) { set_error("vertex %lld is not finite", (long long)v); return RT_EINVAL; }
    xmin = std::min(xmin, x); xmax = std::max(xmax, x); ymin = std::min(ymin, y); ymax = std::max(ymax, y);
  }
  out.nbr.assign(nt, int4{0, 0, 0, 0});
  out.geo.assign(2 * nt, float4{0, 0, 0, 0});
  out.area.assign(nt, 0.0);
  std::vector<int32_t> link(3 * nt, -1);
  std::unordered_map<uint64_t, int64_t> edges;
  edges.reserve((size_t)(nt * 2));
  double min_ratio = INFINITY;
  for (int64_t t = 0; t < nt; ++t) {
    int32_t a[3] = {T[3 * t], T[3 * t + 1], T[3 * t + 2]};
    for (int e = 0; e < 3; ++e)
      if (a[e] < 0 || a[e] >= nv) { set_error("triangle %lld: vertex id out of range", (long long)t); return RT_EINVAL; }
    if (a[0] == a[1] || a[1] == a[2] || a[0] == a[2]) { set_error("triangle %lld is degenerate", (long long)t); return RT_EINVAL; }
    const double ax = V[2 * a[0]], ay = V[2 * a[0] + 1];
    const double bx = V[2 * a[1]], by = V[2 * a[1] + 1];
    const double cx = V[2 * a[2]], cy = V[2 * a[2] + 1];
    const double A = 0.5 * ((bx - ax) * (cy - ay) - (by - ay) * (cx - ax));
    if (!(A > 0.0)) { set_error("triangle %lld is not counter-clockwise (area %g)", (long long)t, A); return RT_EINVAL; }
    out.area[t] = A;
    double P = 0.0;
    for (int e = 0; e < 3; ++e) {
      const int32_t p = a[e], q = a[(e + 1) % 3];
      P += std::hypot(V[2 * q] - V[2 * p], V[2 * q + 1] - V[2 * p + 1]);
      const uint64_t key = ((uint64_t)(uint32_t)std::min(p, q) << 32) | (uint32_t)std::max(p, q);
      auto it = edges.find(key);
      if (it == edges.end()) {
        edges.emplace(key, 3 * t + e);
      } else {
        const int64_t other = it->second;
        if (other < 0) { set_error("edge shared by more than two triangles"); return RT_EINVAL; }
        const int64_t ot = other / 3;
        const int oe = (int)(other % 3);
        if (T[3 * ot + oe] != q) { set_error("triangles %lld and %lld have inconsistent orientation", (long long)ot, (long long)t); return RT_EINVAL; }
        link[3 * t + e] = (int32_t)ot;
        link[other] = (int32_t)t;
        it->second = -1;
      }
    }
    min_ratio = std::min(min_ratio, 2.0 * A / P);
  }
  out.min_2a_over_p = min_ratio;
  std::vector<double> cen(2 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int c = 0; c < 2; ++c)
      cen[2 * t + c] = (V[2 * T[3 * t] + c] + V[2 * T[3 * t + 1] + c] + V[2 * T[3 * t + 2] + c]) / 3.0;
  out.geo2.assign(3 * nt, float4{0, 0, 0, 0});
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t a[3] = {T[3 * t], T[3 * t + 1], T[3 * t + 2]};
    const double A = out.area[t];
    int32_t nb[3];
    float ax[3], ay[3], rx[3], ry[3], dx[3] = {0, 0, 0}, dy[3] = {0, 0, 0};
    for (int e = 0; e < 3; ++e) {
      const int32_t p = a[e], q = a[(e + 1) % 3];
      const double px = V[2 * p], py = V[2 * p + 1], qx = V[2 * q], qy = V[2 * q + 1];
      // outward normal times length of edge p->q for a counter-clockwise triangle
      const double nlx = qy - py, nly = -(qx - px);
      ax[e] = (float)(nlx / A);
      ay[e] = (float)(nly / A);
      rx[e] = (float)(0.5 * (px + qx) - cen[2 * t]);
      ry[e] = (float)(0.5 * (py + qy) - cen[2 * t + 1]);
      if (link[3 * t + e] >= 0) {
        nb[e] = link[3 * t + e];
        dx[e] = (float)(cen[2 * (int64_t)nb[e]] - cen[2 * t]);
        dy[e] = (float)(cen[2 * (int64_t)nb[e] + 1] - cen[2 * t + 1]);
      } else {
        const double mx = 0.5 * (px + qx), my = 0.5 * (py + qy);
        const double dist[4] = {std::fabs(mx - xmin), std::fabs(mx - xmax), std::fabs(my - ymin), std::fabs(my - ymax)};
        int side = 0;
        for (int s = 1; s < 4; ++s)
          if (dist[s] < dist[side]) side = s;
        nb[e] = -1 - side;
      }
    }
    out.nbr[t] = int4{nb[0], nb[1], nb[2], (int)(cell_mat[t] & 255) | ((int)(cell_reg[t] & 255) << 8)};
    out.geo[2 * t] = float4{ax[0], ay[0], ax[1], ay[1]};
    const double eps = A * A * A;   // the limiter's epsilon = K A^3 with K = 1
    out.geo[2 * t + 1] = float4{ax[2], ay[2], (float)A, (float)(eps * eps)};
    out.geo2[3 * t] = float4{rx[0], ry[0], rx[1], ry[1]};
    out.geo2[3 * t + 1] = float4{rx[2], ry[2], dx[0], dy[0]};
    out.geo2[3 * t + 2] = float4{dx[1], dy[1], dx[2], dy[2]};
  }
  return RT_OK;
}

// Device order of the triangles: Morton (Z-order) of the centroids on a
// 2^16 x 2^16 grid over the bounding box, ties by the caller's index. Cells that
// share an edge are then mostly close in the order, so the neighbour rows a
// kernel gathers were read recently by the CTAs working next to it (the caller's
// order may put a neighbour a whole grid row away). perm[new] = caller's index;
// the device arrays of tm (neighbours, geometry) are rewritten in that order
// with neighbour ids renumbered; tm.area stays in the caller's order.
static void reorder_triangles(const rt_mesh* m, TriMeta& tm, std::vector<int32_t>& perm) {
  const int64_t nt = m->n_tri;
  const double* V = m->vxy;
  const int32_t* T = m->tri;
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  std::vector<double> cx(nt), cy(nt);
  for (int64_t t = 0; t < nt; ++t) {
    cx[t] = (V[2 * T[3 * t]] + V[2 * T[3 * t + 1]] + V[2 * T[3 * t + 2]]) / 3.0;
    cy[t] = (V[2 * T[3 * t] + 1] + V[2 * T[3 * t + 1] + 1] + V[2 * T[3 * t + 2] + 1]) / 3.0;
    xmin = std::min(xmin, cx[t]); xmax = std::max(xmax, cx[t]);
    ymin = std::min(ymin, cy[t]); ymax = std::max(ymax, cy[t]);
  }
  const double sx = xmax > xmin ? 65535.0 / (xmax - xmin) : 0.0, sy = ymax > ymin ? 65535.0 / (ymax - ymin) : 0.0;
  auto spread = [](uint32_t v) {   // bit i of v to bit 2i
    uint64_t x = v & 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
  };
  std::vector<uint64_t> key(nt);
  for (int64_t t = 0; t < nt; ++t) {
    const uint32_t ix = (uint32_t)std::min(65535.0, std::max(0.0, (cx[t] - xmin) * sx));
    const uint32_t iy = (uint32_t)std::min(65535.0, std::max(0.0, (cy[t] - ymin) * sy));
    key[t] = (spread(ix) | (spread(iy) << 1)) << 31 | (uint64_t)t;   // ties by the caller's index
  }
  std::vector<uint64_t> order(key);
  std::sort(order.begin(), order.end());
  perm.resize(nt);
  std::vector<int32_t> rank(nt);
  for (int64_t i = 0; i < nt; ++i) {
    perm[i] = (int32_t)(order[i] & 0x7fffffffu);
    rank[perm[i]] = (int32_t)i;
  }
  std::vector<int4> nbr(nt);
  std::vector<float4> geo(2 * nt), geo2(3 * nt);
  for (int64_t i = 0; i < nt; ++i) {
    const int64_t t = perm[i];
    int4 r = tm.nbr[t];
    r.x = r.x >= 0 ? rank[r.x] : r.x;
    r.y = r.y >= 0 ? rank[r.y] : r.y;
    r.z = r.z >= 0 ? rank[r.z] : r.z;
    nbr[i] = r;
    geo[2 * i] = tm.geo[2 * t];
    geo[2 * i + 1] = tm.geo[2 * t + 1];
    for (int j = 0; j < 3; ++j) geo2[3 * i + j] = tm.geo2[3 * t + j];
  }
  tm.nbr.swap(nbr);
  tm.geo.swap(geo);
  tm.geo2.swap(geo2);
}

// ---------------------------------------------------------------- chunk halos
// Halo of each chunk of kTriStgChunk consecutive cells of the device order
// (the staged first-order triangle kernel): the cells outside the chunk that
// share an edge with one of its cells, sorted, padded per chunk to a multiple of
// 4 ids (16-byte copies), and per cell the slots of its neighbours among the
// chunk's staged rows. The staged kernel is used (I.uni = 1, I.ly = the largest
// halo rounded up to 4) when every halo has at most kMaxChunkHalo cells.
constexpr int kMaxChunkHalo = 128;

static void build_chunk_halos(const TriMeta& tm, int64_t n_cells, Instance& I, std::vector<int2>& oc,
                              std::vector<int32_t>& halo, std::vector<uint32_t>& lidx) {
  constexpr int C = kTriStgChunk;
  const int64_t n_chunks = (n_cells + C - 1) / C;
  oc.assign(n_chunks, int2{0, 0});
  halo.clear();
  lidx.assign(n_chunks * C, 0xffffffffu);
  int hmax = 0;
  std::vector<int32_t> h;
  for (int64_t k = 0; k < n_chunks; ++k) {
    const int64_t c0 = k * C, c1 = std::min(n_cells, c0 + C);
    h.clear();
    for (int64_t c = c0; c < c1; ++c) {
      const int nb[3] = {tm.nbr[c].x, tm.nbr[c].y, tm.nbr[c].z};
      for (int e = 0; e < 3; ++e)
        if (nb[e] >= 0 && (nb[e] < c0 || nb[e] >= c1)) h.push_back(nb[e]);
    }
    std::sort(h.begin(), h.end());
    h.erase(std::unique(h.begin(), h.end()), h.end());
    if ((int)h.size() > kMaxChunkHalo) {   // too wide for the staged kernel's buffers
      oc.clear(); halo.clear(); lidx.clear();
      I.uni = 0;
      I.staged_ok = 0;
      return;
    }
    hmax = std::max(hmax, (int)h.size());
    oc[k] = int2{(int)halo.size(), (int)h.size()};
    for (int64_t c = c0; c < c1; ++c) {
      const int nb[3] = {tm.nbr[c].x, tm.nbr[c].y, tm.nbr[c].z};
      uint32_t v = 0;
      for (int e = 0; e < 3; ++e) {
        uint32_t slot = 255;
        if (nb[e] >= c0 && nb[e] < c1) {
          slot = (uint32_t)(nb[e] - c0);
        } else if (nb[e] >= 0) {
          slot = (uint32_t)C + (uint32_t)(std::lower_bound(h.begin(), h.end(), nb[e]) - h.begin());
        }
        v |= slot << (8 * e);
      }
      lidx[c] = v;
    }
    halo.insert(halo.end(), h.begin(), h.end());
    while (halo.size() % 4) halo.push_back(0);
  }
  I.uni = 1;
  I.staged_ok = 1;
  I.ly = (hmax + 3) & ~3;
}

// ---------------------------------------------------------------- tiles
// Ordinates per lane: the largest V in {4, 2, 1} that divides M_pad/32 and for
// which every group of V consecutive ordinates has one sign of xi (zero-weight
// padding ordinates have xi = 0 and fit either sign).
static int choose_cart_vec(const rt_quadrature* quad, int Mpad) {
  for (int V = 4; V >= 2; V /= 2) {
    if ((Mpad / 32) % V != 0) continue;
    bool ok = true;
    for (int g0 = 0; g0 < quad->M && ok; g0 += V) {
      int sgn = 0;
      for (int k = g0; k < std::min<int64_t>(g0 + V, quad->M); ++k) {
        const int sk = quad->xi[k] > 0 ? 1 : (quad->xi[k] < 0 ? -1 : 0);
        if (sk == 0) continue;
        if (sgn == 0) sgn = sk;
        else if (sgn != sk) ok = false;
      }
    }
    if (ok) return V;
  }
  return 1;
}

// Chunk-uniform check: for chunks of 32V ordinates, every chunk has one sign of
// xi and one of eta (zeros fit either). Fills the per-chunk directions.
static bool chunks_uniform(const rt_quadrature* quad, int Mpad, int V, int8_t* dx, int8_t* dy) {
  const int C = 32 * V;
  if (Mpad % C != 0 || Mpad / C > kMaxUniChunks) return false;
  for (int c = 0; c < Mpad / C; ++c) {
    int sx = 0, sy = 0;
    for (int k = c * C; k < std::min<int64_t>((int64_t)(c + 1) * C, quad->M); ++k) {
      const int kx = quad->xi[k] > 0 ? 1 : (quad->xi[k] < 0 ? -1 : 0);
      const int ky = quad->eta[k] > 0 ? 1 : (quad->eta[k] < 0 ? -1 : 0);
      if (kx != 0) {
        if (sx == 0) sx = kx;
        else if (sx != kx) return false;
      }
      if (ky != 0) {
        if (sy == 0) sy = ky;
        else if (sy != ky) return false;
      }
    }
    dx[c] = (int8_t)(sx < 0 ? -1 : 1);
    dy[c] = (int8_t)(sy < 0 ? -1 : 1);
  }
  return true;
}

// Resident CTAs per SM of the Cartesian stage kernel at segment length ly: the
// kernel's launch bound (2 with 8 values per thread and row, else 3) and its shared
// memory (the Heun stage 2 ring is the largest).
static int cart_ctas_per_sm(const Instance& I, int ly) {
  const int by_regs = I.run * I.cvec >= 8 ? 2 : 3;
  const int stage_hi = I.integrator == RT_HEUN ? STAGE_HEUN2 : STAGE_EULER;
  const size_t smem = cart_smem_bytes(I.order, I.storage, I.run, I.cvec, ly, stage_hi) + 1024;
  const int by_smem = (int)((size_t)228 * 1024 / smem);
  return std::max(1, std::min(by_regs, by_smem));
}

// Ordinates regrouped by direction quadrant (xi >= 0 and eta >= 0 first, then
// the quadrants in azimuth order; zeros count as positive), each quadrant padded
// with zero-weight ordinates to whole chunks of C = 128 (or 64) ordinates, when
// the caller's order does not already give sign-uniform chunks and the padding
// costs at most 1/8 more ordinates. Then the chunk-uniform Cartesian kernel
// applies to any quadrature whose quadrants are about chunk-sized multiples
// (the tessellation rule of Sec. 5.1.1, for instance). Fills the regrouped
// arrays (pads: xi = eta = w = 0) and the maps; false: keep the caller's order.
static bool regroup_quadrature(const rt_quadrature* quad, std::vector<double>& xi, std::vector<double>& eta,
                               std::vector<double>& w, std::vector<int32_t>& kmap, std::vector<int32_t>& inv) {
  const int M = (int)quad->M;
  const int Mpad = (M + 31) / 32 * 32;
  int8_t dx[kMaxUniChunks], dy[kMaxUniChunks];
  for (int V = 4; V >= 2; V /= 2)
    if (Mpad % (32 * V) == 0 && chunks_uniform(quad, Mpad, V, dx, dy)) return false;   // already uniform
  auto quadrant = [&](int k) {
    const bool xp = quad->xi[k] >= 0.0, yp = quad->eta[k] >= 0.0;
    return xp ? (yp ? 0 : 3) : (yp ? 1 : 2);
  };
  int count[4] = {0, 0, 0, 0};
  for (int k = 0; k < M; ++k) ++count[quadrant(k)];
  for (int C : {128, 64}) {
    int total = 0;
    for (int q = 0; q < 4; ++q) total += (count[q] + C - 1) / C * C;
    if (total > Mpad + Mpad / 8 || total / C > kMaxUniChunks) continue;
    xi.assign(total, 0.0);
    eta.assign(total, 0.0);
    w.assign(total, 0.0);
    kmap.assign(M, -1);
    inv.assign(total, -1);
    int base = 0;
    for (int q = 0; q < 4; ++q) {
      int slot = base;
      for (int k = 0; k < M; ++k)
        if (quadrant(k) == q) {
          xi[slot] = quad->xi[k];
          eta[slot] = quad->eta[k];
          w[slot] = quad->w[k];
          kmap[k] = slot;
          inv[slot] = k;
          ++slot;
        }
      base += (count[q] + C - 1) / C * C;
    }
    return true;
  }
  return false;
}

static void choose_cart_tiles(Instance& I, int tile_y) {
  I.tx = cart_tile_width(I.run);
  I.n_strips = (I.nx + I.tx - 1) / I.tx;
  int ly = tile_y;
  if (ly <= 0) {
    // Segment length by a throughput model: a CTA pulls n_chunks * (ly + H + 1)
    // rows per work item plus a fixed cost of about 4 rows (tile set-up,
    // epilogue); the block scheduler keeps (resident CTAs per SM x SMs) items in
    // flight, and the last item of a slot adds about one item time. Take the ly
    // in [8, 64] with the least items x item time / slots + item time (ties: the
    // longer segment).
    const int sms = device_sm_count();
    const int chunks = std::max(1, I.Mpad / (32 * I.cvec));
    double best = 0.0;
    ly = 8;
    for (int cand = 8; cand <= 64; ++cand) {
      const int64_t items = (int64_t)I.n_strips * ((I.ny + cand - 1) / cand);
      const int64_t slots = (int64_t)sms * cart_ctas_per_sm(I, cand);
      const double t_item = chunks * (double)(std::min(cand, I.ny) + I.order + 1) + 4.0;
      const double cost = (double)items * t_item / (double)std::min(items, slots) + t_item;
      if (cand == 8 || cost <= best) {
        best = cost;
        ly = cand;
      }
    }
  }
  ly = std::max(1, std::min(ly, 256));
  I.ly = ly;
  I.n_segs = (I.ny + ly - 1) / ly;
}

static void cell_range_items(int64_t n_cells, std::vector<WorkItem>& items) {
  const int sms = device_sm_count();
  int64_t per = (n_cells + 4LL * sms - 1) / (4LL * sms);
  per = std::max<int64_t>(64, std::min<int64_t>(per, 1024));
  per = (per + 7) / 8 * 8;
  const int64_t n = (n_cells + per - 1) / per;
  items.clear();
  for (int64_t i = 0; i < n; ++i) {
    WorkItem w{};
    w.inst = 0;
    w.a = (int32_t)(i * per);
    w.b = (int32_t)std::min<int64_t>(per, n_cells - i * per);
    w.item = (int32_t)i;
    w.count = (int32_t)n;
    items.push_back(w);
  }
}

// ---------------------------------------------------------------- QoI boxes
// Face records of the QoI boxes (Sec. 3.1 QoI-1/2) on a Cartesian grid: for each
// box, its x- side (inside column i_lo, rows j_lo..j_hi-1), x+ side (column
// i_hi-1), y- side (row j_lo, columns i_lo..i_hi-1) and y+ side (row j_hi-1), in
// that order; per face {inside cell, outside cell, the inside cell's other
// neighbour along the normal, box | side << 8}.
static rt_status build_box_faces(const rt_mesh* mesh, const rt_materials* mat, std::vector<int4>& faces) {
  faces.clear();
  if (mat->n_boxes == 0) return RT_OK;
  if (mat->n_boxes < 0 || mat->n_boxes > RT_MAX_BOXES) { set_error("n_boxes must be in 0..%d", RT_MAX_BOXES); return RT_EINVAL; }
  if (!mat->boxes) { set_error("boxes is NULL"); return RT_EINVAL; }
  if (mesh->kind != RT_MESH_CARTESIAN) { set_error("QoI boxes need a Cartesian mesh"); return RT_EINVAL; }
  const int nx = mesh->nx;
  for (int b = 0; b < mat->n_boxes; ++b) {
    int lim[4];
    for (int e = 0; e < 4; ++e) {
      const double v = mat->boxes[4 * b + e];
      const double o = e < 2 ? mesh->x0 : mesh->y0, h = e < 2 ? mesh->dx : mesh->dy;
      const int n = e < 2 ? mesh->nx : mesh->ny;
      if (!std::isfinite(v)) { set_error("box %d: edge %d is not finite", b, e); return RT_EINVAL; }
      const double r = std::nearbyint((v - o) / h);
      if (std::fabs(o + r * h - v) > 1e-9 * std::max(1.0, std::fabs(v)) || r < 1 || r > n - 1) {
        set_error("box %d: edge %g is not a grid line strictly inside the domain", b, v);
        return RT_EINVAL;
      }
      lim[e] = (int)r;
    }
    const int i0 = lim[0], i1 = lim[1], j0 = lim[2], j1 = lim[3];
    if (i1 <= i0 || j1 <= j0) { set_error("box %d: need x_lo < x_hi and y_lo < y_hi", b); return RT_EINVAL; }
    auto cell = [&](int i, int j) { return (int32_t)((int64_t)j * nx + i); };
    for (int j = j0; j < j1; ++j) faces.push_back(make_int4(cell(i0, j), cell(i0 - 1, j), cell(i0 + 1, j), b | 0 << 8));
    for (int j = j0; j < j1; ++j) faces.push_back(make_int4(cell(i1 - 1, j), cell(i1, j), cell(i1 - 2, j), b | 1 << 8));
    for (int i = i0; i < i1; ++i) faces.push_back(make_int4(cell(i, j0), cell(i, j0 - 1), cell(i, j0 + 1), b | 2 << 8));
    for (int i = i0; i < i1; ++i) faces.push_back(make_int4(cell(i, j1 - 1), cell(i, j1), cell(i, j1 - 2), b | 3 << 8));
  }
  return RT_OK;
}

// ---------------------------------------------------------------- build
rt_status build_instance(const rt_mesh* mesh, const rt_materials* mat, const rt_quadrature* quad,
                         const rt_boundary* bc, int order, int integrator, int storage, double dt_target,
                         double t_end, int tile_x, int tile_y, DeviceArena& arena, cudaStream_t stream,
                         Instance& I, std::vector<std::vector<char>>& keep, int variant, int vec) {
  if (!mesh) { set_error("mesh is NULL"); return RT_EINVAL; }
  int64_t n_cells = 0;
  if (mesh->kind == RT_MESH_CARTESIAN) {
    if (mesh->nx < 1 || mesh->ny < 1 || !(mesh->dx > 0) || !(mesh->dy > 0) || !std::isfinite(mesh->dx) || !std::isfinite(mesh->dy)) {
      set_error("Cartesian mesh: need nx, ny >= 1 and dx, dy > 0"); return RT_EINVAL;
    }
    n_cells = (int64_t)mesh->nx * mesh->ny;
    if (n_cells > 0x7fffffffLL) { set_error("Cartesian mesh too large"); return RT_EINVAL; }
  } else if (mesh->kind == RT_MESH_TRIANGLES) {
    n_cells = mesh->n_tri;
  } else {
    set_error("unknown mesh kind %d", mesh->kind); return RT_EINVAL;
  }
  rt_status s = validate_common(mat, quad, bc, order, integrator, storage, t_end, n_cells);
  if (s != RT_OK) return s;
  if (mesh->kind == RT_MESH_TRIANGLES)
    for (int sd = 0; sd < 4; ++sd)
      if (bc->side_kind[sd] == RT_BC_PERIODIC) {
        set_error("periodic sides are supported on Cartesian meshes only"); return RT_EINVAL;
      }
  std::vector<int4> box_faces;
  if ((s = build_box_faces(mesh, mat, box_faces)) != RT_OK) return s;
  if (std::isnan(dt_target)) { set_error("dt is not a number"); return RT_EINVAL; }

  I.kind = mesh->kind; I.order = order; I.integrator = integrator; I.storage = storage;
  I.n_cells = n_cells;
  I.M = (int32_t)quad->M;
  // Cartesian meshes: ordinates regrouped by quadrant when that gives sign-uniform
  // chunks; from here on `quad` is the internal layout (I.M stays the caller's count)
  std::vector<double> rq_xi, rq_eta, rq_w;
  std::vector<int32_t> rq_kmap, rq_inv;
  rt_quadrature rq{};
  I.regrouped = 0;
  if (mesh->kind == RT_MESH_CARTESIAN && variant != 1 &&
      regroup_quadrature(quad, rq_xi, rq_eta, rq_w, rq_kmap, rq_inv)) {
    rq.M = (int64_t)rq_xi.size();
    rq.xi = rq_xi.data();
    rq.eta = rq_eta.data();
    rq.w = rq_w.data();
    quad = &rq;
    I.regrouped = 1;
  }
  I.Mpad = (int32_t)((quad->M + 31) / 32 * 32);
  // ordinates per lane of the cell-range and triangle kernels: 32*vec divides Mpad
  I.vec = (I.Mpad % 128 == 0) ? 4 : ((I.Mpad % 64 == 0) ? 2 : 1);
  I.t_end = t_end;
  I.n_regions = mat->n_regions;
  const size_t es = storage == RT_BF16 ? 2 : 4;
  if (I.kind == RT_MESH_CARTESIAN) {
    I.nx = mesh->nx; I.ny = mesh->ny;
  }

  // --- triangles: mesh metadata
  TriMeta tm;
  std::vector<int2> stg_halo_oc;
  std::vector<int32_t> stg_halo;
  std::vector<uint32_t> stg_lidx;
  if (I.kind == RT_MESH_TRIANGLES) {
    s = triangle_metadata(mesh, mat->cell_mat, mat->cell_region, tm);
    if (s != RT_OK) return s;
    reorder_triangles(mesh, tm, I.cell_perm);
  }

  // --- time step (Sec. 4.3: uniform dt = T / N_t)
  double dtt = dt_target;
  if (!(dtt > 0.0)) {
    dtt = (I.kind == RT_MESH_CARTESIAN) ? 0.5 * std::min(mesh->dx, mesh->dy) : 0.9 * tm.min_2a_over_p;
  }
  I.n_steps = steps_for(t_end, dtt);
  I.dt = t_end / (double)I.n_steps;

  // --- source rate 2 pi sum A Q (reported as source_int = t * rate)
  double wsum = 0.0;
  for (int64_t k = 0; k < quad->M; ++k) wsum += quad->w[k];
  double aq = 0.0;
  if (I.kind == RT_MESH_CARTESIAN) {
    for (int64_t i = 0; i < n_cells; ++i) aq += mat->Q[mat->cell_mat[i]];
    aq *= mesh->dx * mesh->dy;
  } else {
    for (int64_t i = 0; i < n_cells; ++i) aq += tm.area[i] * mat->Q[mat->cell_mat[i]];
  }
  I.source_rate = aq * wsum;

  // --- tiles and work items
  int8_t cdx[kMaxUniChunks] = {0}, cdy[kMaxUniChunks] = {0};
  if (I.kind == RT_MESH_CARTESIAN) {
    if (variant < 0 || variant > 2) { set_error("variant must be 0, 1 or 2"); return RT_EINVAL; }
    // per-lane width first; the chunk-uniform variant is taken (automatically) when
    // the same width also gives sign-uniform chunks, or when asked for
    if (vec != 0 && vec != 1 && vec != 2 && vec != 4) { set_error("vec must be 0, 1, 2 or 4"); return RT_EINVAL; }
    I.uni = 0;
    I.cvec = choose_cart_vec(quad, I.Mpad);
    if (vec != 0) {
      if (vec > I.cvec) { set_error("vec %d: the quadrature allows at most %d ordinates per lane", vec, I.cvec); return RT_EINVAL; }
      I.cvec = vec;
    }
    if (tile_x != 0 && tile_x != 16 && tile_x != 32) { set_error("tile_x must be 0, 16 or 32"); return RT_EINVAL; }
    I.run = 2;
    // 32-cell strips (runs of 4 cells per warp) with chunk-uniform directions and
    // 2 ordinates per lane: fewer face evaluations and shared-memory reads per
    // cell, but twice the chunks of 4 ordinates per lane. Chosen automatically
    // only when 4 ordinates per lane do not give uniform chunks (the 16-cell
    // strips with 4 per lane measured faster where both apply), and only on
    // grids of more than kWideMinCells cells: with 256 ordinates (quadrants of
    // 64) the per-lane kernel measured faster on 70^2..280^2 grids (0.16 against
    // 0.21 ms per step at 70^2, 0.31 against 0.34 at 280^2), the 32-cell strips
    // on 560^2 (0.64 against 0.68) and 1400^2 (2.31 against 2.89).
    constexpr int64_t kWideMinCells = 100000;
    bool wide = false;
    if (variant != 1 && (vec == 0 || vec == 2) && tile_x != 16) {
      const bool narrow4 = tile_x == 0 && vec == 0 && I.cvec >= 4 && chunks_uniform(quad, I.Mpad, 4, cdx, cdy);
      const bool small = tile_x == 0 && variant == 0 && vec == 0 && n_cells <= kWideMinCells;
      wide = !narrow4 && !small && chunks_uniform(quad, I.Mpad, 2, cdx, cdy);
    }
    if (wide) {
      I.uni = 1;
      I.cvec = 2;
      I.run = 4;
    } else if (tile_x == 32) {
      set_error("tile_x 32 needs chunk-uniform directions with 2 ordinates per lane");
      return RT_EINVAL;
    } else if (variant != 1) {
      for (int V = (variant == 2 && vec == 0 ? 4 : I.cvec); V >= 2; V /= 2) {
        if (chunks_uniform(quad, I.Mpad, V, cdx, cdy)) {
          I.uni = 1;
          I.cvec = V;
          break;
        }
        if (variant == 0 || vec != 0) break;
      }
      if (variant == 2 && !I.uni) {
        set_error("variant 2 needs every ordinate chunk to have one sign of xi and one of eta");
        return RT_EINVAL;
      }
    }
    choose_cart_tiles(I, tile_y);
    I.stage_items.clear();
    const int n = I.n_strips * I.n_segs;
    for (int g = 0; g < I.n_segs; ++g)
      for (int st = 0; st < I.n_strips; ++st) {
        WorkItem w{};
        w.inst = 0; w.a = st; w.b = g; w.item = (int32_t)I.stage_items.size(); w.count = n;
        I.stage_items.push_back(w);
      }
    const int stage_hi = integrator == RT_HEUN ? STAGE_HEUN2 : STAGE_EULER;
    I.cart_smem = cart_smem_bytes(order, storage, I.run, I.cvec, I.ly, stage_hi);
    if (I.cart_smem > 227 * 1024) { set_error("tile %dx%d needs %zu bytes of shared memory", I.tx, I.ly, I.cart_smem); return RT_EINVAL; }
  } else {
    // persistent work items: item g processes 64-cell chunks g, g + G, ...; the
    // staged first-order kernel runs two CTAs per SM, the others three
    const int64_t n_chunks = (n_cells + 63) / 64;
    if (order == 1) {
      build_chunk_halos(tm, n_cells, I, stg_halo_oc, stg_halo, stg_lidx);
      // the staged kernel's two row buffers must fit the shared memory of a CTA
      const int top = integrator == RT_HEUN ? STAGE_HEUN2 : STAGE_EULER;
      if (I.staged_ok && tri_staged_smem_bytes(I.vec, storage, I.ly, top) > 108 * 1024) {
        I.uni = 0;
        I.staged_ok = 0;
        stg_halo_oc.clear(); stg_halo.clear(); stg_lidx.clear();
      }
    }
    const int G = (int)std::min<int64_t>(n_chunks, (I.uni ? 2LL : 3LL) * device_sm_count());
    I.stage_items.clear();
    for (int g = 0; g < G; ++g) {
      WorkItem w{};
      w.inst = 0; w.a = g; w.b = G; w.item = g; w.count = G;
      I.stage_items.push_back(w);
    }
  }
  cell_range_items(n_cells, I.init_items);

  // --- device buffers
  const size_t psi_bytes = (size_t)n_cells * I.Mpad * es;
  void* p = nullptr;
  for (int b = 0; b < 2; ++b) {
    if ((s = arena.get(psi_bytes, &p)) != RT_OK) return s;
    I.psi[b] = p;
    if ((s = arena.get((size_t)n_cells * 4, &p)) != RT_OK) return s;
    I.phi[b] = (float*)p;
  }
  if ((s = arena.get(sizeof(InstState), &p)) != RT_OK) return s;
  I.st = (InstState*)p;
  const size_t n_part = std::max(I.stage_items.size(), I.init_items.size());
  if ((s = arena.get(n_part * NQ * sizeof(double), &p)) != RT_OK) return s;
  I.partials = (double*)p;
  // QoI boxes: tasks = (face, block of 128 ordinates holding an ordinate that
  // leaves through the face, by the sign the kernel sees: FP32 omega . n > 0),
  // in work items of kBoxTasksPerItem tasks
  I.n_boxes = mat->n_boxes;
  I.box_items.clear();
  int4* d_faces = nullptr;
  double* d_box_part = nullptr;
  std::vector<int4> box_tasks;
  if (!box_faces.empty()) {
    std::vector<int> leave[4];
    for (int sd = 0; sd < 4; ++sd)
      for (int kb = 0; kb * 128 < I.Mpad; ++kb) {
        bool any = false;
        for (int k = kb * 128; k < std::min<int64_t>((int64_t)kb * 128 + 128, quad->M); ++k) {
          const float dir = (float)(sd < 2 ? quad->xi[k] : quad->eta[k]);
          any = any || ((sd & 1) ? dir : -dir) > 0.f;
        }
        if (any) leave[sd].push_back(kb);
      }
    for (const int4& f : box_faces)
      for (int kb : leave[(f.w >> 8) & 3]) box_tasks.push_back(make_int4(f.x, f.y, f.z, f.w | kb << 12));
  }
  if (!box_tasks.empty()) {
    const int nt = (int)box_tasks.size();
    const int n_it = (nt + kBoxTasksPerItem - 1) / kBoxTasksPerItem;
    for (int g = 0; g < n_it; ++g) {
      WorkItem w{};
      w.inst = 0; w.a = g * kBoxTasksPerItem; w.b = std::min(kBoxTasksPerItem, nt - w.a);
      w.item = g; w.count = n_it;
      I.box_items.push_back(w);
    }
    keep.emplace_back(box_tasks.size() * sizeof(int4));
    std::memcpy(keep.back().data(), box_tasks.data(), box_tasks.size() * sizeof(int4));
    if ((s = arena.get(box_tasks.size() * sizeof(int4), &p)) != RT_OK) return s;
    d_faces = (int4*)p;
    RT_CUDA_TRY(cudaMemcpyAsync(d_faces, keep.back().data(), box_tasks.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                stream));
    if ((s = arena.get((size_t)n_it * 2 * kMaxBox * sizeof(double), &p)) != RT_OK) return s;
    d_box_part = (double*)p;
    RT_CUDA_TRY(cudaMemsetAsync(d_box_part, 0, (size_t)n_it * 2 * kMaxBox * sizeof(double), stream));
  }

  // host images of per-cell and per-ordinate data (kept alive until the stream syncs)
  keep.emplace_back(3 * (size_t)I.Mpad * sizeof(float));
  float* hq = reinterpret_cast<float*>(keep.back().data());
  for (int k = 0; k < I.Mpad; ++k) {
    const bool in = k < quad->M;
    hq[k] = in ? (float)quad->xi[k] : 0.f;
    hq[I.Mpad + k] = in ? (float)quad->eta[k] : 0.f;
    hq[2 * I.Mpad + k] = in ? (float)quad->w[k] : 0.f;
  }
  float* d_quad = nullptr;
  if ((s = arena.get(3 * (size_t)I.Mpad * sizeof(float), &p)) != RT_OK) return s;
  d_quad = (float*)p;
  RT_CUDA_TRY(cudaMemcpyAsync(d_quad, hq, 3 * (size_t)I.Mpad * sizeof(float), cudaMemcpyHostToDevice, stream));
  I.kmap = I.inv = nullptr;
  if (I.regrouped) {
    // caller <-> internal ordinate maps for psi input and output
    keep.emplace_back(((size_t)I.M + I.Mpad) * sizeof(int32_t));
    int32_t* hm = reinterpret_cast<int32_t*>(keep.back().data());
    for (int k = 0; k < I.M; ++k) hm[k] = rq_kmap[k];
    for (int k = 0; k < I.Mpad; ++k) hm[I.M + k] = k < (int)rq_inv.size() ? rq_inv[k] : -1;
    if ((s = arena.get(((size_t)I.M + I.Mpad) * sizeof(int32_t), &p)) != RT_OK) return s;
    I.kmap = (int32_t*)p;
    I.inv = I.kmap + I.M;
    RT_CUDA_TRY(cudaMemcpyAsync(I.kmap, hm, ((size_t)I.M + I.Mpad) * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  }

  uint8_t* d_mat = nullptr;
  uint8_t* d_reg = nullptr;
  int4* d_nbr = nullptr;
  float4* d_geo = nullptr;
  float4* d_geo2 = nullptr;
  float* d_lg = nullptr;
  int2* d_halo_oc = nullptr;
  int32_t* d_halo = nullptr;
  uint32_t* d_lidx = nullptr;
  if (I.kind == RT_MESH_CARTESIAN) {
    keep.emplace_back(2 * (size_t)n_cells);
    uint8_t* hm = reinterpret_cast<uint8_t*>(keep.back().data());
    for (int64_t i = 0; i < n_cells; ++i) {
      hm[i] = (uint8_t)mat->cell_mat[i];
      hm[n_cells + i] = (uint8_t)mat->cell_region[i];
    }
    if ((s = arena.get(2 * (size_t)n_cells, &p)) != RT_OK) return s;
    d_mat = (uint8_t*)p;
    d_reg = d_mat + n_cells;
    RT_CUDA_TRY(cudaMemcpyAsync(d_mat, hm, 2 * (size_t)n_cells, cudaMemcpyHostToDevice, stream));
  } else {
    keep.emplace_back(n_cells * sizeof(int4));
    std::memcpy(keep.back().data(), tm.nbr.data(), n_cells * sizeof(int4));
    const void* hn = keep.back().data();
    keep.emplace_back(2 * n_cells * sizeof(float4));
    std::memcpy(keep.back().data(), tm.geo.data(), 2 * n_cells * sizeof(float4));
    const void* hg = keep.back().data();
    if ((s = arena.get(n_cells * sizeof(int4), &p)) != RT_OK) return s;
    d_nbr = (int4*)p;
    if ((s = arena.get(2 * n_cells * sizeof(float4), &p)) != RT_OK) return s;
    d_geo = (float4*)p;
    RT_CUDA_TRY(cudaMemcpyAsync(d_nbr, hn, n_cells * sizeof(int4), cudaMemcpyHostToDevice, stream));
    RT_CUDA_TRY(cudaMemcpyAsync(d_geo, hg, 2 * n_cells * sizeof(float4), cudaMemcpyHostToDevice, stream));
    if (I.staged_ok) {
      // staged first-order kernel: chunk halos and neighbour slots
      const size_t b_oc = stg_halo_oc.size() * sizeof(int2), b_h = stg_halo.size() * sizeof(int32_t),
                   b_l = stg_lidx.size() * sizeof(uint32_t);
      keep.emplace_back(b_oc + b_h + b_l);
      char* hk = keep.back().data();
      std::memcpy(hk, stg_halo_oc.data(), b_oc);
      std::memcpy(hk + b_oc, stg_halo.data(), b_h);
      std::memcpy(hk + b_oc + b_h, stg_lidx.data(), b_l);
      if ((s = arena.get(b_oc, &p)) != RT_OK) return s;
      d_halo_oc = (int2*)p;
      if ((s = arena.get(std::max<size_t>(b_h, 16), &p)) != RT_OK) return s;
      d_halo = (int32_t*)p;
      if ((s = arena.get(b_l, &p)) != RT_OK) return s;
      d_lidx = (uint32_t*)p;
      RT_CUDA_TRY(cudaMemcpyAsync(d_halo_oc, hk, b_oc, cudaMemcpyHostToDevice, stream));
      if (b_h) RT_CUDA_TRY(cudaMemcpyAsync(d_halo, hk + b_oc, b_h, cudaMemcpyHostToDevice, stream));
      RT_CUDA_TRY(cudaMemcpyAsync(d_lidx, hk + b_oc + b_h, b_l, cudaMemcpyHostToDevice, stream));
    }
    if (order == 2) {
      keep.emplace_back(3 * n_cells * sizeof(float4));
      std::memcpy(keep.back().data(), tm.geo2.data(), 3 * n_cells * sizeof(float4));
      if ((s = arena.get(3 * n_cells * sizeof(float4), &p)) != RT_OK) return s;
      d_geo2 = (float4*)p;
      RT_CUDA_TRY(cudaMemcpyAsync(d_geo2, keep.back().data(), 3 * n_cells * sizeof(float4), cudaMemcpyHostToDevice,
                                  stream));
      const size_t lg_bytes = (size_t)n_cells * 2 * I.Mpad * sizeof(float);
      if ((s = arena.get(lg_bytes, &p)) != RT_OK) return s;
      d_lg = (float*)p;
      RT_CUDA_TRY(cudaMemsetAsync(d_lg, 0, lg_bytes, stream));
    }
  }
  for (int b = 0; b < 2; ++b) {
    RT_CUDA_TRY(cudaMemsetAsync(I.psi[b], 0, psi_bytes, stream));
    RT_CUDA_TRY(cudaMemsetAsync(I.phi[b], 0, (size_t)n_cells * 4, stream));
  }
  RT_CUDA_TRY(cudaMemsetAsync(I.st, 0, sizeof(InstState), stream));
  RT_CUDA_TRY(cudaMemsetAsync(I.partials, 0, n_part * NQ * sizeof(double), stream));

  // --- descriptor
  InstDesc& D = I.desc;
  std::memset(&D, 0, sizeof(D));
  if (I.kind == RT_MESH_CARTESIAN) {
    for (int b = 0; b < 2; ++b)
      if ((s = encode_psi_map(&D.tm_psi_halo[b], I.psi[b], storage, I.Mpad, I.nx, I.ny, 32 * I.cvec,
                              I.tx + 2 * order)) != RT_OK) return s;
    if ((s = encode_psi_map(&D.tm_psi_center, I.psi[0], storage, I.Mpad, I.nx, I.ny, 32 * I.cvec, I.tx)) != RT_OK)
      return s;
  }
  for (int b = 0; b < 2; ++b) { D.psi[b] = I.psi[b]; D.phi[b] = I.phi[b]; }
  D.mat = d_mat; D.region = d_reg;
  D.xi = d_quad; D.eta = d_quad + I.Mpad; D.w = d_quad + 2 * I.Mpad;
  D.tri_nbr = d_nbr; D.tri_geo = d_geo;
  D.tri_geo2 = d_geo2; D.tri_lg = d_lg;
  D.tri_halo_oc = d_halo_oc; D.tri_halo = d_halo; D.tri_lidx = d_lidx;
  D.tri_hmax = (I.kind == RT_MESH_TRIANGLES && I.staged_ok) ? I.ly : 0;
  D.st = I.st; D.partials = I.partials;
  D.kind = I.kind; D.order = order; D.integrator = integrator; D.storage = storage;
  D.nx = I.nx; D.ny = I.ny; D.M = I.M; D.Mpad = I.Mpad;
  D.n_chunks = (I.kind == RT_MESH_CARTESIAN) ? I.Mpad / (32 * I.cvec) : I.Mpad / kChunk; D.tx = I.tx; D.ly = I.ly; D.n_strips = I.n_strips;
  D.n_segs = I.n_segs; D.n_items = (int32_t)I.stage_items.size(); D.n_regions = I.n_regions;
  D.n_cells = n_cells; D.n_steps = I.n_steps;
  D.wait_limit = 4000000000LL;   // about two seconds of SM clock
  D.drop_load = -1;
  if (I.kind == RT_MESH_CARTESIAN) {
    D.inv_dx = (float)(1.0 / mesh->dx); D.inv_dy = (float)(1.0 / mesh->dy);
    D.dx_d = mesh->dx; D.dy_d = mesh->dy; D.area_d = mesh->dx * mesh->dy;
  }
  D.dt = (float)I.dt; D.dt_d = I.dt;
  for (int sd = 0; sd < 4; ++sd) D.ghost[sd] = bc->side_kind[sd] == RT_BC_INFLOW ? (float)bc->inflow[sd] : 0.f;
  D.periodic_x = bc->side_kind[0] == RT_BC_PERIODIC ? 1 : 0;
  D.periodic_y = bc->side_kind[2] == RT_BC_PERIODIC ? 1 : 0;
  D.uni = I.uni;
  for (int c = 0; c < kMaxUniChunks; ++c) {
    D.cdir_x[c] = cdx[c];
    D.cdir_y[c] = cdy[c];
  }
  for (int m = 0; m < kMaxMat; ++m) {
    const bool in = m < mat->n_mat;
    const double sa = in ? mat->sigma_a[m] : 0.0, ss = in ? mat->sigma_s[m] : 0.0, q = in ? mat->Q[m] : 0.0;
    D.sig_t[m] = (float)(sa + ss);
    D.sig_s2pi[m] = (float)(ss / (2.0 * M_PI));
    D.q_src[m] = (float)q;
    D.sig_a[m] = sa;
    D.sig_a_f[m] = (float)sa;
  }
  D.box_tasks = d_faces;
  D.box_partials = d_box_part;
  D.n_boxes = I.n_boxes;
  D.n_box_tasks = (int32_t)box_tasks.size();
  I.device_bytes = arena.bytes;
  return RT_OK;
}

rt_status launch_step(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int kind, int integrator,
                      int storage, int order, int run, int cvec, int ly_max, int vec, cudaStream_t stream,
                      int uni, const WorkItem* d_box_items, int n_box_items) {
  const int stages[2] = {integrator == RT_HEUN ? STAGE_HEUN1 : STAGE_EULER, STAGE_HEUN2};
  const int n_st = integrator == RT_HEUN ? 2 : 1;
  for (int i = 0; i < n_st; ++i) {
    cudaError_t e;
    if (kind == RT_MESH_CARTESIAN)
      e = launch_cart_stage(d_desc, d_items, n_items, stages[i], order, storage, run, cvec, ly_max, stream, uni);
    else if (order == 2)
      e = launch_tri2_stage(d_desc, d_items, n_items, stages[i], storage, std::min(vec, 2), vec, stream);
    else if (uni)
      e = launch_tri_staged(d_desc, d_items, n_items, stages[i], storage, vec, ly_max, stream);
    else
      e = launch_tri_stage(d_desc, d_items, n_items, stages[i], storage, vec, stream);
    if (e != cudaSuccess) {
      set_error("stage launch failed: %s", cudaGetErrorString(e));
      return RT_ECUDA;
    }
  }
  // QoI boxes: one launch after the step's last stage
  if (n_box_items > 0) {
    cudaError_t e = launch_box_outflow(d_desc, d_box_items, n_box_items, stages[n_st - 1], storage, stream);
    if (e != cudaSuccess) {
      set_error("box outflow launch failed: %s", cudaGetErrorString(e));
      return RT_ECUDA;
    }
  }
  return RT_OK;
}

rt_status launch_init_all(const InstDesc* d_desc, const WorkItem* d_init_items, int n_init_items,
                          const WorkItem* d_box_items, int n_box_items, int vec, int storage, cudaStream_t stream) {
  cudaError_t e = launch_init(d_desc, d_init_items, n_init_items, vec, storage, stream);
  if (e == cudaSuccess && n_box_items > 0)
    e = launch_box_outflow(d_desc, d_box_items, n_box_items, STAGE_INIT, storage, stream);
  if (e != cudaSuccess) {
    set_error("init launch failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  return RT_OK;
}

rt_status prepare_instance_kernels(const Instance& I, int ly_max) {
  const int stages[2] = {I.integrator == RT_HEUN ? STAGE_HEUN1 : STAGE_EULER, STAGE_HEUN2};
  if (I.kind != RT_MESH_CARTESIAN) {
    if (!I.staged_ok) return RT_OK;
    for (int i = 0; i < (I.integrator == RT_HEUN ? 2 : 1); ++i) {
      cudaError_t e = prepare_tri_staged(stages[i], I.storage, I.vec, ly_max);
      if (e != cudaSuccess) {
        set_error("kernel set-up failed: %s", cudaGetErrorString(e));
        return RT_ECUDA;
      }
    }
    return RT_OK;
  }
  for (int i = 0; i < (I.integrator == RT_HEUN ? 2 : 1); ++i) {
    cudaError_t e = prepare_cart_stage(stages[i], I.order, I.storage, I.run, I.cvec, ly_max, I.uni);
    if (e != cudaSuccess) {
      set_error("kernel set-up failed: %s", cudaGetErrorString(e));
      return RT_ECUDA;
    }
  }
  return RT_OK;
}

rt_status read_inst_state(const Instance& I, cudaStream_t stream, InstState* h) {
  RT_CUDA_TRY(cudaMemcpyAsync(h, I.st, sizeof(InstState), cudaMemcpyDeviceToHost, stream));
  RT_CUDA_TRY(cudaStreamSynchronize(stream));
  if (h->status == DEV_TIMEOUT) {
    set_error("a device-side wait ran out (block %lld, load %lld)", (long long)(h->timeout_where >> 32),
              (long long)(h->timeout_where & 0xffffffff));
    return RT_ETIMEOUT;
  }
  if (h->status == DEV_NONFINITE) {
    set_error("the solution became non-finite by step %lld", (long long)h->step);
    return RT_ENONFINITE;
  }
  return RT_OK;
}

void fill_qoi(const Instance& I, const InstState& h, rt_qoi_t* out) {
  std::memset(out, 0, sizeof(*out));
  out->step = h.step;
  out->n_steps = I.n_steps;
  out->t = (double)h.step * I.dt;
  out->n_regions = I.n_regions;
  out->status = h.status;
  for (int r = 0; r < I.n_regions; ++r) {
    out->abs_now[r] = h.S_cur[r];
    out->abs_int[r] = h.I[r];
  }
  out->mass = h.S_cur[kQMass];
  out->outflow_now = h.S_cur[kQOut];
  out->outflow_int = h.I[kQOut];
  out->source_int = out->t * I.source_rate;
  out->n_boxes = I.n_boxes;
  for (int b = 0; b < I.n_boxes; ++b) {
    out->box_out_now[b] = h.B_cur[b];
    out->box_out_int[b] = h.B_I[b];
  }
}

static int64_t convert_chunk(const Instance& I) {
  return std::max<int64_t>(1, std::min<int64_t>(I.n_cells, (64LL << 20) / (8LL * I.M)));
}

rt_status copy_psi_out(const Instance& I, DeviceArena& arena, cudaStream_t stream, int buf, double* host) {
  const size_t es = I.storage == RT_BF16 ? 2 : 4;
  const int64_t chunk = convert_chunk(I);
  void* tmp = nullptr;
  rt_status st = arena.get((size_t)chunk * I.M * 8, &tmp);
  if (st != RT_OK) return st;
  // cells in device order; with a cell permutation each chunk is staged on the
  // host and its rows scattered to the caller's order
  const bool perm = !I.cell_perm.empty();
  std::vector<double> stage(perm ? (size_t)chunk * I.M : 0);
  for (int64_t c0 = 0; c0 < I.n_cells; c0 += chunk) {
    const int64_t nc = std::min(chunk, I.n_cells - c0);
    const char* src = (const char*)I.psi[buf] + (size_t)c0 * I.Mpad * es;
    cudaError_t e = launch_convert_out(src, (double*)tmp, nc, I.M, I.Mpad, I.storage, I.kmap, stream);
    double* out = perm ? stage.data() : host + c0 * I.M;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, (size_t)nc * I.M * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess && perm)
      for (int64_t i = 0; i < nc; ++i)
        std::memcpy(host + (int64_t)I.cell_perm[c0 + i] * I.M, stage.data() + i * I.M, (size_t)I.M * 8);
    if (e != cudaSuccess) {
      arena.release(tmp);
      set_error("reading psi failed: %s", cudaGetErrorString(e));
      return RT_ECUDA;
    }
  }
  arena.release(tmp);
  return RT_OK;
}

rt_status copy_psi_in(const Instance& I, DeviceArena& arena, cudaStream_t stream, int buf, const double* host) {
  const size_t es = I.storage == RT_BF16 ? 2 : 4;
  const int64_t chunk = convert_chunk(I);
  void* tmp = nullptr;
  rt_status st = arena.get((size_t)chunk * I.M * 8, &tmp);
  if (st != RT_OK) return st;
  const bool perm = !I.cell_perm.empty();
  std::vector<double> stage(perm ? (size_t)chunk * I.M : 0);
  for (int64_t c0 = 0; c0 < I.n_cells; c0 += chunk) {
    const int64_t nc = std::min(chunk, I.n_cells - c0);
    char* dst = (char*)I.psi[buf] + (size_t)c0 * I.Mpad * es;
    if (perm)
      for (int64_t i = 0; i < nc; ++i)
        std::memcpy(stage.data() + i * I.M, host + (int64_t)I.cell_perm[c0 + i] * I.M, (size_t)I.M * 8);
    const double* in = perm ? stage.data() : host + c0 * I.M;
    cudaError_t e = cudaMemcpyAsync(tmp, in, (size_t)nc * I.M * 8, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = launch_convert_in((const double*)tmp, dst, nc, I.M, I.Mpad, I.storage, I.inv, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      arena.release(tmp);
      set_error("writing psi failed: %s", cudaGetErrorString(e));
      return RT_ECUDA;
    }
  }
  arena.release(tmp);
  return RT_OK;
}

rt_status copy_psi_cells_out(const Instance& I, DeviceArena& arena, cudaStream_t stream, int buf,
                             const int64_t* cells, int64_t n, double* host) {
  if (n == 0) return RT_OK;
  // device index of each caller's cell
  std::vector<int64_t> dev((size_t)n);
  std::vector<int32_t> rank;
  if (!I.cell_perm.empty()) {
    rank.resize(I.cell_perm.size());
    for (size_t i = 0; i < I.cell_perm.size(); ++i) rank[I.cell_perm[i]] = (int32_t)i;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (cells[i] < 0 || cells[i] >= I.n_cells) { set_error("cell id %lld out of range", (long long)cells[i]); return RT_EINVAL; }
    dev[i] = rank.empty() ? cells[i] : rank[cells[i]];
  }
  const size_t es = I.storage == RT_BF16 ? 2 : 4;
  const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(n, (16LL << 20) / (8LL * I.M)));
  void* tmp = nullptr;
  rt_status st = arena.get((size_t)batch * I.M * 8, &tmp);
  if (st != RT_OK) return st;
  for (int64_t c0 = 0; c0 < n; c0 += batch) {
    const int64_t nc = std::min(batch, n - c0);
    cudaError_t e = cudaSuccess;
    for (int64_t i = 0; i < nc && e == cudaSuccess; ++i) {
      const char* src = (const char*)I.psi[buf] + (size_t)dev[c0 + i] * I.Mpad * es;
      e = launch_convert_out(src, (double*)tmp + i * I.M, 1, I.M, I.Mpad, I.storage, I.kmap, stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host + c0 * I.M, tmp, (size_t)nc * I.M * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      arena.release(tmp);
      set_error("reading psi of cells failed: %s", cudaGetErrorString(e));
      return RT_ECUDA;
    }
  }
  arena.release(tmp);
  return RT_OK;
}

}  // namespace rtk
