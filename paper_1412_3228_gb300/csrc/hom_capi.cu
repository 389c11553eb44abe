// Library-wide services of the C ABI: error strings, FFT plan cache, solver workspace, the
// effective-stiffness reduction and resource release.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "hom_internal.h"
#include "hom_fast2d.h"
#include "hom_plan.h"

namespace hom {

static thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

bool grid_supported(int n) {
  std::vector<int> r;
  return n >= 3 && n <= kMaxN && factorize(n, r) && (int)r.size() <= kMaxStages;
}

namespace {

struct DevicePlan {
  Plan plan{};
  void* mem = nullptr;  // perm + twiddles in one allocation
};

struct DeviceCache {
  std::map<std::pair<int, int>, DevicePlan> plans;  // by (n, max_radix)
  void* ws = nullptr;
  size_t ws_bytes = 0;
};

std::mutex g_mutex;
std::map<int, DeviceCache> g_cache;  // by device ordinal

DeviceCache& cache_for_current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_cache[dev];
}

}  // namespace

int get_plan(int n, int max_radix, Plan* out) {
  std::lock_guard<std::mutex> lk(g_mutex);
  DeviceCache& dc = cache_for_current_device();
  auto it = dc.plans.find(std::make_pair(n, max_radix));
  if (it != dc.plans.end()) {
    *out = it->second.plan;
    return HOM_OK;
  }
  HostPlan hp;
  if (!build_host_plan(n, hp, max_radix) || (int)hp.radix.size() > kMaxStages)
    return set_error(HOM_ERR_UNSUPPORTED_SIZE, "grid size %d has a prime factor above 13", n);
  std::vector<unsigned char> host(plan_table_bytes(n), 0);
  fill_plan_tables(hp, host.data());
  DevicePlan dp;
  cudaError_t e = cudaMalloc(&dp.mem, host.size());
  if (e != cudaSuccess) return set_error(HOM_ERR_OOM, "plan allocation failed: %s", cudaGetErrorString(e));
  e = cudaMemcpy(dp.mem, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dp.mem);
    return set_error(HOM_ERR_CUDA, "plan upload failed: %s", cudaGetErrorString(e));
  }
  Plan& p = dp.plan;
  p.n = n;
  p.nstage = (int)hp.radix.size();
  for (int s = 0; s < p.nstage; ++s) {
    p.radix[s] = hp.radix[s];
    p.span[s] = hp.span[s];
  }
  plan_dividers(p);
  set_plan_pointers(p, static_cast<unsigned char*>(dp.mem));
  dc.plans[std::make_pair(n, max_radix)] = dp;
  *out = p;
  return HOM_OK;
}

int get_workspace(size_t bytes, void** ptr) {
  std::lock_guard<std::mutex> lk(g_mutex);
  DeviceCache& dc = cache_for_current_device();
  if (bytes > dc.ws_bytes) {
    if (dc.ws) {
      cudaDeviceSynchronize();
      cudaFree(dc.ws);
      dc.ws = nullptr;
      dc.ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&dc.ws, bytes);
    if (e != cudaSuccess) {
      dc.ws = nullptr;
      return set_error(HOM_ERR_OOM, "workspace allocation of %zu bytes failed: %s", bytes,
                       cudaGetErrorString(e));
    }
    dc.ws_bytes = bytes;
  }
  *ptr = dc.ws;
  return HOM_OK;
}

}  // namespace hom

using namespace hom;

extern "C" const char* hom_last_error(void) { return g_last_error.c_str(); }

extern "C" int32_t hom_version(void) { return 100; }

extern "C" int32_t hom_build_flags(void) {
#ifdef HOM_DEBUG
  return HOM_BUILD_DEBUG;
#else
  return 0;
#endif
}

extern "C" void hom_release(void) {
  std::lock_guard<std::mutex> lk(g_mutex);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_cache) {
    cudaSetDevice(kv.first);
    cudaDeviceSynchronize();
    for (auto& p : kv.second.plans) cudaFree(p.second.mem);
    if (kv.second.ws) cudaFree(kv.second.ws);
  }
  g_cache.clear();
  release_backward_buffers();
  release_graphs();
  fast2d_release();
  cudaSetDevice(cur);
}

extern "C" int hom_effective_stiffness(int32_t ncells, int32_t dim, const double* E, const double* mean_sigma,
                                       double* C_out) {
  if (ncells <= 0 || (dim != 2 && dim != 3) || !E || !mean_sigma || !C_out)
    return set_error(HOM_ERR_INVALID_ARG, "hom_effective_stiffness: invalid arguments");
  const int nc = nc_of(dim);
  const size_t cnt = (size_t)ncells * nc * nc;
  std::vector<double> S(cnt);
  cudaPointerAttributes attr{};
  bool dev = cudaPointerGetAttributes(&attr, mean_sigma) == cudaSuccess && attr.type == cudaMemoryTypeDevice;
  cudaGetLastError();
  if (dev) {
    HOM_CUDA_TRY(cudaMemcpy(S.data(), mean_sigma, cnt * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(S.data(), mean_sigma, cnt * sizeof(double));
  }
  // For each cell: C E^T = S^T, i.e. E C^T = S: solve with Gaussian elimination (rows = loads).
  for (int c = 0; c < ncells; ++c) {
    double A[36], X[36];
    std::memcpy(A, E + (size_t)c * nc * nc, sizeof(double) * nc * nc);
    std::memcpy(X, S.data() + (size_t)c * nc * nc, sizeof(double) * nc * nc);
    // partial-pivot elimination on [A | X]
    for (int k = 0; k < nc; ++k) {
      int piv = k;
      for (int r = k + 1; r < nc; ++r)
        if (std::fabs(A[r * nc + k]) > std::fabs(A[piv * nc + k])) piv = r;
      if (!(std::fabs(A[piv * nc + k]) > 0.0))
        return set_error(HOM_ERR_INVALID_ARG, "hom_effective_stiffness: load cases of cell %d are singular", c);
      if (piv != k)
        for (int j = 0; j < nc; ++j) {
          std::swap(A[k * nc + j], A[piv * nc + j]);
          std::swap(X[k * nc + j], X[piv * nc + j]);
        }
      for (int r = 0; r < nc; ++r) {
        if (r == k) continue;
        const double f = A[r * nc + k] / A[k * nc + k];
        for (int j = 0; j < nc; ++j) {
          A[r * nc + j] -= f * A[k * nc + j];
          X[r * nc + j] -= f * X[k * nc + j];
        }
      }
    }
    // X now holds C^T row k scaled by A[k][k]
    double* Cc = C_out + (size_t)c * nc * nc;
    for (int k = 0; k < nc; ++k)
      for (int j = 0; j < nc; ++j) Cc[j * nc + k] = X[k * nc + j] / A[k * nc + k];
  }
  return HOM_OK;
}
