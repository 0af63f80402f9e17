// lst_noalloc.cu -- mini-doublet finder that performs no device allocation at call time.
//
// Who needs this: code that must not call cudaMalloc/cudaFree while it runs. Examples are
// a host framework that owns all device memory through its own caching allocator (a
// foreign cudaFree synchronises the whole device and defeats that allocator), trigger or
// real-time loops where the implicit synchronisation of cudaMalloc/cudaFree would break a
// latency budget, and code that enqueues work while another thread holds a global-mode
// stream capture (cudaMalloc is prohibited then). Such callers bring their own input and
// output buffers; the only intermediate storage here is the fixed array below.
//
// The scratch (hits grouped by sensor, the sensor histogram and offsets, counters) is one
// file-scope __device__ array of LST_NOALLOC_SCRATCH_BYTES. Every GPU that loads the
// library holds it until the process exits. Every call uses the same array and leaves its
// contents behind; each call clears the parts that must start at zero. Two calls whose
// work overlaps on the GPU (different streams, or different host threads) race on it and
// give wrong results: serialise them.
#include <mutex>

#include "lst_internal.cuh"

namespace lstk {
bool ctx_geometry(lst_ctx ctx, DevGeom *g, lst_cuts *c, int *device);
void set_last_error(const char *msg);
}

namespace {

using namespace lstk;

constexpr int64_t NA_MAX_HITS = LST_NOALLOC_MAX_HITS;
constexpr int64_t NA_MAX_SENSORS = LST_NOALLOC_MAX_SENSORS;
// byte layout of the scratch array
constexpr size_t NA_OFF_HIT = 0;                                        // float4 [MAX_HITS]
constexpr size_t NA_OFF_ORIG = NA_OFF_HIT + 16 * NA_MAX_HITS;          // int32  [MAX_HITS]
constexpr size_t NA_OFF_CNT = NA_OFF_ORIG + 4 * NA_MAX_HITS;           // int32  [MAX_SENSORS]
constexpr size_t NA_OFF_SOFF = NA_OFF_CNT + 4 * NA_MAX_SENSORS;        // int32  [MAX_SENSORS + 1]
constexpr size_t NA_OFF_CTR = NA_OFF_SOFF + 4 * (NA_MAX_SENSORS + 64); // counters (below)
constexpr size_t NA_BYTES = NA_OFF_CTR + 256;
static_assert(NA_BYTES == LST_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");
enum { NA_MDCOUNT = 0, NA_FLAGS = 2 };   // counter words: [0..1] unsigned long long MD count, [2] flags

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

struct NaScratch {
  float4 *hit;
  int32_t *orig, *cnt, *soff, *ctr;
};

__host__ __device__ NaScratch na_view(unsigned char *base) {
  NaScratch s;
  s.hit = reinterpret_cast<float4 *>(base + NA_OFF_HIT);
  s.orig = reinterpret_cast<int32_t *>(base + NA_OFF_ORIG);
  s.cnt = reinterpret_cast<int32_t *>(base + NA_OFF_CNT);
  s.soff = reinterpret_cast<int32_t *>(base + NA_OFF_SOFF);
  s.ctr = reinterpret_cast<int32_t *>(base + NA_OFF_CTR);
  return s;
}

__global__ void k_na_clear(unsigned char *base, int n_sensors) {
  NaScratch s = na_view(base);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_sensors; i += gridDim.x * blockDim.x) s.cnt[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 64) s.ctr[threadIdx.x] = 0;
}

__global__ void k_na_count(unsigned char *base, const float *x, const float *y, const float *z,
                           const int32_t *sensor, int n, int n_sensors) {
  NaScratch s = na_view(base);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int id = sensor[i];
    if (id < 0 || id >= n_sensors || !isfinite(x[i]) || !isfinite(y[i]) || !isfinite(z[i])) {
      atomicOr(s.ctr + NA_FLAGS, 1);
      continue;
    }
    atomicAdd(s.cnt + id, 1);
  }
}

// exclusive scan of the histogram by one CTA; re-zeroes the histogram as scatter cursor
__global__ void k_na_scan(unsigned char *base, int n_sensors) {
  NaScratch s = na_view(base);
  const int per = (n_sensors + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  int local = 0;
  for (int k = 0; k < per && b0 + k < n_sensors; k++) local += s.cnt[b0 + k];
  __shared__ int s_w[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int inc = warp_incl_scan(local);
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int v = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0;
    const int vi = warp_incl_scan(v);
    if (lane < (int)(blockDim.x >> 5)) s_w[lane] = vi - v;
  }
  __syncthreads();
  int run = s_w[wid] + inc - local;
  for (int k = 0; k < per && b0 + k < n_sensors; k++) {
    const int c = s.cnt[b0 + k];
    s.soff[b0 + k] = run;
    s.cnt[b0 + k] = 0;
    run += c;
  }
  if (b0 < n_sensors && b0 + per >= n_sensors) s.soff[n_sensors] = run;
}

__global__ void k_na_scatter(unsigned char *base, const float *x, const float *y, const float *z,
                             const int32_t *sensor, int n, int n_sensors) {
  NaScratch s = na_view(base);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int id = sensor[i];
    const float xi = x[i], yi = y[i], zi = z[i];
    if (id < 0 || id >= n_sensors || !isfinite(xi) || !isfinite(yi) || !isfinite(zi)) continue;
    const int pos = s.soff[id] + atomicAdd(s.cnt + id, 1);
    s.hit[pos] = make_float4(xi, yi, zi, sqrtf(xi * xi + yi * yi));
    s.orig[pos] = i;
  }
}

// One warp per module (static striding). Passing pairs are compacted by ballot and written
// with one atomic per warp and 32 candidates straight into the caller's output.
__global__ void k_na_md(unsigned char *base, DevGeom g, lst_cuts c, int32_t *out_hits, float *out_kappa,
                        long long capacity) {
  NaScratch s = na_view(base);
  if (s.ctr[NA_FLAGS]) return;
  unsigned long long *md_count = reinterpret_cast<unsigned long long *>(s.ctr + NA_MDCOUNT);
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < g.n_mod; m += warps) {
    const int lo0 = s.soff[2 * m], lo1 = s.soff[2 * m + 1], up1 = s.soff[2 * m + 2];
    const int nlo = lo1 - lo0, nup = up1 - lo1;
    const long long np = (long long)nlo * nup;
    const bool endcap = g.subdet[m] != 0;
    for (long long b = 0; b < np; b += 32) {
      const long long p = b + lane;
      bool pass = false;
      float k = 0.0f;
      int i = 0, j = 0;
      if (p < np) {
        i = (int)(p / nup);
        j = (int)(p - (long long)i * nup);
        pass = md_cut(s.hit[lo0 + i], s.hit[lo1 + j], endcap, c, k);
      }
      const unsigned bal = __ballot_sync(FULL, pass);
      if (bal == 0) continue;
      unsigned long long base_out = 0;
      if (lane == 0) base_out = atomicAdd(md_count, (unsigned long long)__popc(bal));
      base_out = __shfl_sync(FULL, base_out, 0);
      if (pass) {
        const unsigned long long o = base_out + __popc(bal & lanemask_lt());
        if ((long long)o < capacity) {
          out_hits[2 * o] = s.orig[lo0 + i];
          out_hits[2 * o + 1] = s.orig[lo1 + j];
          if (out_kappa) out_kappa[o] = k;
        }
      }
    }
  }
}

__global__ void k_na_finish(unsigned char *base, int64_t *md_count_out) {
  NaScratch s = na_view(base);
  const unsigned long long n = *reinterpret_cast<unsigned long long *>(s.ctr + NA_MDCOUNT);
  *md_count_out = s.ctr[NA_FLAGS] ? -1 : (int64_t)n;
}

// Device address of the scratch array and the SM count, looked up once per device (with
// that device current).
std::mutex g_na_mutex;
unsigned char *g_na_ptr[64] = {nullptr};
int g_na_sms[64] = {0};

lst_status na_setup(int device, unsigned char **out, int *sms, const char **why) {
  std::lock_guard<std::mutex> lk(g_na_mutex);
  if (device < 0 || device >= 64) { *why = "device ordinal above 63"; return LST_ERR_ARG; }
  if (!g_na_ptr[device]) {
    void *p = nullptr;
    int n_sm = 0;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess || !p || n_sm <= 0) {
      *why = e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address or no SMs";
      return LST_ERR_CUDA;
    }
    g_na_ptr[device] = static_cast<unsigned char *>(p);
    g_na_sms[device] = n_sm;
  }
  *out = g_na_ptr[device];
  *sms = g_na_sms[device];
  return LST_OK;
}

}  // namespace

extern "C" lst_status lst_find_minidoublets_noalloc(lst_ctx ctx, const float *x, const float *y, const float *z,
                                                    const int32_t *sensor, int64_t n_hits, int32_t *md_hits,
                                                    float *md_kappa, int64_t capacity, int64_t *md_count,
                                                    void *cuda_stream) {
  DevGeom g;
  lst_cuts c;
  int device = 0;
  auto reject = [](lst_status s, const char *msg) { lstk::set_last_error(msg); return s; };
  if (!ctx || !md_count) return reject(LST_ERR_ARG, "null ctx or md_count");
  if (!lstk::ctx_geometry(ctx, &g, &c, &device)) return reject(LST_ERR_NOT_READY, "no geometry loaded");
  if (n_hits < 0 || n_hits > NA_MAX_HITS)
    return reject(LST_ERR_ARG, "n_hits outside 0..LST_NOALLOC_MAX_HITS (524288): the fixed scratch is too small");
  if (2 * (int64_t)g.n_mod > NA_MAX_SENSORS)
    return reject(LST_ERR_ARG, "2*n_mod above LST_NOALLOC_MAX_SENSORS (32768): the fixed scratch is too small");
  if (capacity < 0 || capacity > INT32_MAX) return reject(LST_ERR_ARG, "capacity outside 0..INT32_MAX");
  if (n_hits > 0 && (!x || !y || !z || !sensor)) return reject(LST_ERR_ARG, "null hit array");
  if (capacity > 0 && !md_hits) return reject(LST_ERR_ARG, "null md_hits with capacity > 0");
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return reject(LST_ERR_CUDA, cudaGetErrorString(e));
  if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return reject(LST_ERR_CUDA, cudaGetErrorString(e));
  unsigned char *base = nullptr;
  int sms = 0;
  const char *why = nullptr;
  lst_status st = na_setup(device, &base, &sms, &why);
  if (st == LST_OK) {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int ns = 2 * g.n_mod, n = (int)n_hits;
    const int grid = 2 * sms;   // two 256-thread CTAs per SM for the grid-stride kernels
    k_na_clear<<<grid, 256, 0, s>>>(base, ns);
    k_na_count<<<grid, 256, 0, s>>>(base, x, y, z, sensor, n, ns);
    k_na_scan<<<1, 1024, 0, s>>>(base, ns);
    k_na_scatter<<<grid, 256, 0, s>>>(base, x, y, z, sensor, n, ns);
    k_na_md<<<grid, 256, 0, s>>>(base, g, c, md_hits, md_kappa, (long long)capacity);
    k_na_finish<<<1, 1, 0, s>>>(base, md_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = LST_ERR_CUDA; lstk::set_last_error(cudaGetErrorString(e)); }
  } else {
    lstk::set_last_error(why);
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return st;
}
