// Code handles: validation of a (2,k)-regular parity-check matrix over GF(2^m), the GF(2^m)
// tables and the Fourier index maps (Appendix A), and the device copies the kernels read.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "nbfd_internal.h"

namespace nbfd {

static thread_local char g_err[512] = "";

int set_error(int status, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

int check_cuda(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return NBFD_OK;
  if (e == cudaErrorMemoryAllocation)
    return set_error(NBFD_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(NBFD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// SM count of the current device, looked up once per device (launch sizing runs per launch)
int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev >= 0 && dev < 64) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  n = n > 0 ? n : 1;
  if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// Raises the dynamic shared-memory limit of `kernel` on the current device to `bytes` once, not
// at every launch.
cudaError_t ensure_smem(const void *kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find({kernel, dev});
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
  }
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    size_t &v = done[{kernel, dev}];
    v = v > bytes ? v : bytes;
  }
  return e;
}

// GF(2^m) by the linear-feedback recurrence alpha^{i+1} = alpha * alpha^i mod poly.
// Returns false if poly is not primitive of degree m.
static bool build_field(int m, uint32_t poly, std::vector<int> &exp2q, std::vector<int> &log) {
  const int q = 1 << m;
  if (poly >> (m + 1) != 0 || ((poly >> m) & 1u) == 0) return false;
  exp2q.assign(2 * q, 0);
  log.assign(q, -1);
  int x = 1;
  for (int i = 0; i < q - 1; ++i) {
    if (log[x] != -1) return false;  // order of alpha < q-1
    exp2q[i] = x;
    log[x] = i;
    x <<= 1;
    if (x & q) x ^= static_cast<int>(poly);
  }
  if (x != 1) return false;
  for (int i = q - 1; i < 2 * q; ++i) exp2q[i] = exp2q[i - (q - 1)];
  return true;
}

// Index map z -> H z with H = (A^i)^T, h = alpha^i (Appendix A). A^i is the matrix of
// x -> h*x, so its column j is h * alpha^j and entry (r, j) is bit r of h*alpha^j; hence bit j
// of H z = (A^i)^T z is the parity of z AND (h * alpha^j).
static void build_index_map(int m, const std::vector<int> &gexp, const std::vector<int> &glog,
                            std::vector<uint8_t> &table) {
  const int q = 1 << m;
  table.assign((size_t)q * q, 0);
  for (int h = 1; h < q; ++h) {
    int col[8];
    for (int j = 0; j < m; ++j) col[j] = gexp[glog[h] + j];  // h * alpha^j
    for (int z = 0; z < q; ++z) {
      int img = 0;
      for (int j = 0; j < m; ++j) img |= (__builtin_popcount(z & col[j]) & 1) << j;
      table[(size_t)h * q + z] = static_cast<uint8_t>(img);
    }
  }
}

}  // namespace nbfd

using namespace nbfd;

extern "C" int nbfd_field_index_map(int m, uint32_t prim_poly, uint8_t *table) {
  if (m < 2 || m > 8 || !table) return set_error(NBFD_EINVAL, "m outside [2, 8] or table NULL");
  std::vector<int> gexp, glog;
  if (!build_field(m, prim_poly, gexp, glog))
    return set_error(NBFD_EPOLY, "0x%x is not a primitive polynomial of degree %d", prim_poly, m);
  std::vector<uint8_t> t;
  build_index_map(m, gexp, glog, t);
  memcpy(table, t.data(), t.size());
  return NBFD_OK;
}

extern "C" const char *nbfd_last_error(void) { return g_err; }

extern "C" const char *nbfd_status_string(int s) {
  switch (s) {
    case NBFD_OK: return "NBFD_OK";
    case NBFD_EINVAL: return "NBFD_EINVAL";
    case NBFD_ENOTREG: return "NBFD_ENOTREG";
    case NBFD_EPOLY: return "NBFD_EPOLY";
    case NBFD_EDUP: return "NBFD_EDUP";
    case NBFD_EZERO: return "NBFD_EZERO";
    case NBFD_ENOMEM: return "NBFD_ENOMEM";
    case NBFD_ECUDA: return "NBFD_ECUDA";
    case NBFD_ETIMEDOUT: return "NBFD_ETIMEDOUT";
    case NBFD_EBUSY: return "NBFD_EBUSY";
    case NBFD_ENOTSUP: return "NBFD_ENOTSUP";
    default: return "NBFD_E?";
  }
}

extern "C" int nbfd_code_create(int N, int M, int k, int m, uint32_t prim_poly, int n_edges,
                                const int32_t *edge_check, const int32_t *edge_var,
                                const uint16_t *edge_h, nbfd_code **out) {
  g_err[0] = '\0';
  if (!out) return set_error(NBFD_EINVAL, "out is NULL");
  *out = nullptr;
  if (m < 2 || m > 8) return set_error(NBFD_EINVAL, "m = %d outside [2, 8]", m);
  if (k < 2 || k > 32) return set_error(NBFD_EINVAL, "k = %d outside [2, 32]", k);
  if (N <= 0 || M <= 0) return set_error(NBFD_EINVAL, "N and M must be positive");
  if (!edge_check || !edge_var || !edge_h) return set_error(NBFD_EINVAL, "edge arrays are NULL");
  if ((long long)n_edges != 2LL * N || (long long)n_edges != (long long)M * k)
    return set_error(NBFD_ENOTREG, "n_edges = %d must equal 2N = %lld and M*k = %lld", n_edges,
                     2LL * N, (long long)M * k);
  const int q = 1 << m;
  std::vector<int> gexp, glog;
  if (!build_field(m, prim_poly, gexp, glog))
    return set_error(NBFD_EPOLY, "0x%x is not a primitive polynomial of degree %d", prim_poly, m);

  std::vector<int> deg_c(M, 0), deg_v(N, 0);
  std::set<std::pair<int, int>> seen;
  for (int e = 0; e < n_edges; ++e) {
    const int c = edge_check[e], v = edge_var[e];
    if (c < 0 || c >= M || v < 0 || v >= N)
      return set_error(NBFD_EINVAL, "edge %d = (%d, %d) out of range", e, c, v);
    if (edge_h[e] == 0 || edge_h[e] >= q)
      return set_error(NBFD_EZERO, "edge %d entry %u not in [1, %d)", e, edge_h[e], q);
    if (!seen.insert({c, v}).second)
      return set_error(NBFD_EDUP, "edge (%d, %d) appears twice", c, v);
    ++deg_c[c];
    ++deg_v[v];
  }
  for (int c = 0; c < M; ++c)
    if (deg_c[c] != k) return set_error(NBFD_ENOTREG, "check %d has degree %d != k", c, deg_c[c]);
  for (int v = 0; v < N; ++v)
    if (deg_v[v] != 2) return set_error(NBFD_ENOTREG, "variable %d has degree %d != 2", v, deg_v[v]);

  nbfd_code *code = new (std::nothrow) nbfd_code();
  if (!code) return set_error(NBFD_ENOMEM, "host allocation failed");
  code->N = N;
  code->M = M;
  code->k = k;
  code->m = m;
  code->q = q;
  code->E = n_edges;
  code->poly = prim_poly;
  cudaGetDevice(&code->device);

  // check-major slots: stable sort of the caller's edges by check
  std::vector<int32_t> order(n_edges);
  for (int e = 0; e < n_edges; ++e) order[e] = e;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return edge_check[a] < edge_check[b]; });
  code->caller_edge_of_slot = order;
  std::vector<int32_t> h_edge_var(n_edges), h_var_edges(2 * N, -1);
  std::vector<uint8_t> h_edge_h(n_edges);
  std::vector<int> fill(N, 0);
  for (int s = 0; s < n_edges; ++s) {
    const int e = order[s];
    h_edge_var[s] = edge_var[e];
    h_edge_h[s] = static_cast<uint8_t>(edge_h[e]);
    h_var_edges[2 * edge_var[e] + fill[edge_var[e]]++] = s;
  }

  build_index_map(m, gexp, glog, code->index_map);
  std::vector<uint8_t> h_exp(2 * q), h_log(q, 0);
  for (int i = 0; i < 2 * q; ++i) h_exp[i] = static_cast<uint8_t>(gexp[i]);
  for (int x = 1; x < q; ++x) h_log[x] = static_cast<uint8_t>(glog[x]);

  // Fourier-domain syndrome points of every slot: H_cv alpha^i, i < m (Section 3.2)
  std::vector<uint8_t> h_edge_z(8ull * n_edges, 0);
  for (int s = 0; s < n_edges; ++s)
    for (int i = 0; i < m; ++i)
      h_edge_z[8ull * s + i] = code->index_map[(size_t)h_edge_h[s] * q + (1u << i)];

  // one device block:
  // [edge_var E*4][var_edges 2N*4][edge_h E][perm q*q][exp 2q][log q][edge_z E*8]
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off_ev = 0, off_ve = align(off_ev + 4ull * n_edges), off_eh = align(off_ve + 8ull * N),
         off_pm = align(off_eh + n_edges), off_ex = align(off_pm + (size_t)q * q),
         off_lg = align(off_ex + 2 * q), off_ez = align(off_lg + q),
         total = align(off_ez + 8ull * n_edges);
  cudaError_t err = cudaMalloc(&code->d_block, total);
  if (err != cudaSuccess) {
    delete code;
    return check_cuda(err, "cudaMalloc(code tables)");
  }
  char *b = static_cast<char *>(code->d_block);
  code->d_edge_var = reinterpret_cast<int32_t *>(b + off_ev);
  code->d_var_edges = reinterpret_cast<int32_t *>(b + off_ve);
  code->d_edge_h = reinterpret_cast<uint8_t *>(b + off_eh);
  code->d_perm = reinterpret_cast<uint8_t *>(b + off_pm);
  code->d_gf_exp = reinterpret_cast<uint8_t *>(b + off_ex);
  code->d_gf_log = reinterpret_cast<uint8_t *>(b + off_lg);
  code->d_edge_z = reinterpret_cast<uint8_t *>(b + off_ez);
  std::vector<char> staging(total, 0);
  memcpy(staging.data() + off_ev, h_edge_var.data(), 4ull * n_edges);
  memcpy(staging.data() + off_ve, h_var_edges.data(), 8ull * N);
  memcpy(staging.data() + off_eh, h_edge_h.data(), n_edges);
  memcpy(staging.data() + off_pm, code->index_map.data(), (size_t)q * q);
  memcpy(staging.data() + off_ex, h_exp.data(), 2 * q);
  memcpy(staging.data() + off_lg, h_log.data(), q);
  memcpy(staging.data() + off_ez, h_edge_z.data(), 8ull * n_edges);
  err = cudaMemcpy(code->d_block, staging.data(), total, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    cudaFree(code->d_block);
    delete code;
    return check_cuda(err, "cudaMemcpy(code tables)");
  }
  *out = code;
  return NBFD_OK;
}

extern "C" void nbfd_code_destroy(nbfd_code *code) {
  if (!code) return;
  if (code->d_block) cudaFree(code->d_block);
  delete code;
}

extern "C" int nbfd_code_info(const nbfd_code *code, int *N, int *M, int *k, int *m) {
  if (!code) return set_error(NBFD_EINVAL, "code is NULL");
  if (N) *N = code->N;
  if (M) *M = code->M;
  if (k) *k = code->k;
  if (m) *m = code->m;
  return NBFD_OK;
}

extern "C" int nbfd_code_edge_order(const nbfd_code *code, int32_t *caller_edge_of_slot) {
  if (!code || !caller_edge_of_slot) return set_error(NBFD_EINVAL, "NULL argument");
  memcpy(caller_edge_of_slot, code->caller_edge_of_slot.data(), 4ull * code->E);
  return NBFD_OK;
}

extern "C" int nbfd_code_index_map(const nbfd_code *code, uint8_t *table) {
  if (!code || !table) return set_error(NBFD_EINVAL, "NULL argument");
  memcpy(table, code->index_map.data(), code->index_map.size());
  return NBFD_OK;
}
