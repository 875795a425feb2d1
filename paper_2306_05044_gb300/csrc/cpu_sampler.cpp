// Host (CPU) implementation of both hemisphere samplers wrapped in the GGX
// VNDF routine (the cap sampler also on the extended domain), for the paper's
// CPU benchmark (Sec. 4, "CPU Synthetic
// Benchmark": the sampler called in a loop, median time over 100 runs).
// It is an explicit entry point for host callers, never a fallback of the GPU
// entry points.  Plain portable C++17: FP32 arithmetic written branch-free so
// that the compiler can vectorise the loop (omp simd), the same rounding-aware
// formulas as the CUDA kernels (cancellation-free sin^2 for the cap sampler,
// the rewritten disk lift for the prior one, sin/cos(pi x) from its Taylor
// series), and a persistent pool of host threads for the split across cores.  Where the ISA has a
// fused multiply-add (every AArch64 core) the loop vectorises; on the x86-64
// baseline, which has none, std::fma is a library call and the loop stays
// scalar, with the same results.  -fno-trapping-math lets the compiler compute
// both sides of the domain selects; -ffp-contract=off keeps the compiler from
// fusing a product and a sum that the source writes apart (every fused
// multiply-add here is an explicit std::fma), so the results are the same on
// both ISAs and the extended method equals the upper one above the horizon.
#include <pthread.h>

#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <memory>
#include <mutex>
#include <thread>

#include "vndf.h"

namespace {

constexpr float kPiF = 3.14159265358979323846f;

__attribute__((always_inline)) inline void sincospi_taylor_host(float x, float& s, float& c) {
  // sin/cos(pi r) on r = x - j/2 in [-1/4, 1/4] (exact reduction), Taylor terms to r^9 / r^10;
  // x = 2 u1 is in [0, 2), so j = int(2x + 1/2) is the nearest integer (a conversion, which
  // vectorises on every baseline ISA, unlike rint)
  const int ji = static_cast<int>(2.f * x + 0.5f);
  const float j = static_cast<float>(ji);
  const float r = std::fma(-0.5f, j, x);
  const float r2 = r * r;
  float ps = std::fma(r2, 0.0821458866111282288f, -0.599264529320792077f);
  ps = std::fma(r2, ps, 2.55016403987734549f);
  ps = std::fma(r2, ps, -5.16771278004997003f);
  ps = std::fma(r2, ps, 3.14159265358979323846f);
  ps *= r;
  float pc = std::fma(r2, -0.0258068913900140009f, 0.235330630358893200f);
  pc = std::fma(r2, pc, -1.33526276885458949f);
  pc = std::fma(r2, pc, 4.05871212641676822f);
  pc = std::fma(r2, pc, -4.93480220054467931f);
  pc = std::fma(r2, pc, 1.f);
  const int k = ji & 3;
  const float a = (k & 1) ? pc : ps;
  const float b = (k & 1) ? ps : pc;
  s = (k & 2) ? -a : a;
  c = ((k + 1) & 2) ? -b : b;
}

// Condition-number threshold of the cap sampler's half vector above which a sample is
// recomputed in double precision (the GPU kernels use the same test and threshold).
constexpr float kRescueKappa = 24.f;

template <int METHOD, bool PRECISE = false>
__attribute__((always_inline)) inline void sample_host(float wx, float wy, float wz, float ax, float ay, float u1, float u2, float& mx, float& my,
                        float& mz, float& pdf, bool& bad) {
  constexpr bool kExt = METHOD == VNDF_METHOD_SPHERICAL_CAP_EXTENDED;
  constexpr bool kCap = METHOD != VNDF_METHOD_POLAR_DISK;
  // the upper domain needs wi.z > 0; the extended one 1 + z_i' >= 2^-40, tested once a is formed
  bool ok = (kExt | (wz > 0.f)) & (ax > 0.f) & (ay > 0.f) & std::isfinite(wx) & std::isfinite(wy) &
            std::isfinite(wz) & std::isfinite(ax) & std::isfinite(ay);
  // keep the arithmetic finite on out-of-domain lanes (their results are replaced below)
  wz = ok ? wz : 1.f;
  ax = ok ? ax : 1.f;
  ay = ok ? ay : 1.f;
  wx = ok ? wx : 0.f;
  wy = ok ? wy : 0.f;
  // Sec. 2 step (1): i = M^-1 wi / |M^-1 wi|
  const float sx = ax * wx, sy = ay * wy;
  const float l2 = std::fma(sx, sx, std::fma(sy, sy, wz * wz));
  const float rl = 1.f / std::sqrt(l2);
  const float ix = sx * rl, iy = sy * rl, iz = wz * rl;
  const float rho2 = std::fma(ix, ix, iy * iy);  // 1 - i.z^2
  // a = 1 + i.z; below the horizon rho2 / (1 - i.z), which does not cancel
  float a = 1.f + iz;
  if constexpr (kExt) {
    a = iz < 0.f ? rho2 / (1.f - iz) : a;
    ok &= a >= 0x1p-40f;
  }
  float sp, cp;
  sincospi_taylor_host(2.f * u1, sp, cp);
  float hx, hy, hz;
  if constexpr (kCap) {
    // Sec. 3.3: c on the cap z in (-i.z, 1], h = c + i
    const float st = std::sqrt(u2 * std::fma(2.f * a, 1.f - u2, u2 * rho2));
    hx = std::fma(st, cp, ix);
    hy = std::fma(st, sp, iy);
    hz = (1.f - u2) * a;
  } else {
    // Heitz 2018 cross-section sampler (Sec. 2 step (2))
    const float tmp = rho2;
    const bool pole = !(tmp > 0.f);
    const float rt = 1.f / std::sqrt(pole ? 1.f : tmp);
    const float w1x = pole ? 1.f : -iy * rt, w1y = pole ? 0.f : ix * rt;
    const float w2x = -iz * w1y, w2y = iz * w1x, w2z = std::fma(ix, w1y, -iy * w1x);
    const float r = std::sqrt(u2);
    const float t1 = r * cp, t2o = r * sp;
    const float om = 1.f - u2;
    const float q = std::sqrt(std::fma(u2 * sp, sp, om));
    const float s = 0.5f * a, oms = 0.5f * tmp / a;
    const bool pos = t2o >= 0.f;
    const float big = pos ? q + t2o : q - t2o;
    const float small = om / big;
    const float qm = pos ? small : big, qp = pos ? big : small;
    const float t2 = std::fma(oms, q, s * t2o);
    const float ti = std::sqrt(s * qm * std::fma(2.f * oms, q, s * qp));
    hx = std::fma(t1, w1x, std::fma(t2, w2x, ti * ix));
    hy = std::fma(t1, w1y, std::fma(t2, w2y, ti * iy));
    hz = std::fma(t2, w2z, ti * iz);
  }
  // Sec. 2 step (3) and the fused density of Eq. 1
  const float vx = ax * hx, vy = ay * hy, vz = hz;
  const float vv = std::fma(vx, vx, std::fma(vy, vy, vz * vz));
  const float nv = std::sqrt(vv);
  const float rv = 1.f / nv;
  mx = ok ? vx * rv : 0.f;
  my = ok ? vy * rv : 0.f;
  mz = ok ? vz * rv : 1.f;
  float p;
  if constexpr (kCap) {
    const float hh = std::fma(hx, hx, std::fma(hy, hy, hz * hz));
    // (|v|^2 / |h|^2) |v| / (pi ax ay a): every factor stays in FP32 range (|v|^3 would
    // underflow for tiny roughness on the extended domain's smallest cap heights)
    p = (vv / hh) * nv / (kPiF * ax * ay * a);
  } else {
    const float hi = std::fmax(std::fma(hx, ix, std::fma(hy, iy, hz * iz)), 0.f);
    p = 2.f * hi * vv * nv / (kPiF * ax * ay * a);
  }
  pdf = ok ? p : 0.f;
  bad = false;
  if constexpr (PRECISE && kCap) {
    // |c.x| + |i.x| etc. bound the rounding of h; compare it with |v| and |h|
    const float sx = std::fabs(hx - ix) + std::fabs(ix), sy = std::fabs(hy - iy) + std::fabs(iy);
    const float k2 = std::fma(ax * sx, ax * sx, std::fma(ay * sy, ay * sy, hz * hz));
    const float kh2 = std::fma(sx, sx, std::fma(sy, sy, hz * hz));
    const float hh2 = std::fma(hx, hx, std::fma(hy, hy, hz * hz));
    constexpr float k = kRescueKappa * kRescueKappa;
    bad = ok & ((k2 > k * vv) | (kh2 > k * hh2));
  }
}

// One cap sample in double precision (Sec. 2 steps (1)-(3), Sec. 3.3, the fused density
// of Eq. 1), for the samples sample_host flags; inputs are in the domain.
template <bool EXT>
void sample_host_double(float wx, float wy, float wz, float ax, float ay, float u1, float u2, float& mx, float& my,
                        float& mz, float& pdf) {
  constexpr double kPiD = 3.14159265358979323846;
  const double axd = ax, ayd = ay, u1d = u1, u2d = u2;
  const double sx = axd * wx, sy = ayd * wy, sz = wz;
  const double l = std::sqrt(sx * sx + sy * sy + sz * sz);
  const double ix = sx / l, iy = sy / l, iz = sz / l;
  const double rho2 = ix * ix + iy * iy;
  double a = 1.0 + iz;
  if (EXT && iz < 0.0) a = rho2 / (1.0 - iz);
  const double st = std::sqrt(u2d * (2.0 * a * (1.0 - u2d) + u2d * rho2));
  const double phi = 2.0 * kPiD * u1d;
  const double hx = st * std::cos(phi) + ix, hy = st * std::sin(phi) + iy, hz = (1.0 - u2d) * a;
  const double vx = axd * hx, vy = ayd * hy, vz = hz;
  const double vv = vx * vx + vy * vy + vz * vz, nv = std::sqrt(vv);
  mx = static_cast<float>(vx / nv);
  my = static_cast<float>(vy / nv);
  mz = static_cast<float>(vz / nv);
  const double hh = hx * hx + hy * hy + hz * hz;
  pdf = static_cast<float>((vv / hh) * nv / (kPiD * axd * ayd * a));
}

struct HostArgs {
  const float *wx, *wy, *wz, *ax, *ay, *u1, *u2;
  float *mx, *my, *mz, *pdf;
};

template <int METHOD, bool PDF, bool PRECISE>
void run_range(const HostArgs& h, int64_t i0, int64_t i1) {
  const float* ay = h.ay ? h.ay : h.ax;
  constexpr int64_t kBlock = 2048;  // samples per pass: the vector loop, then the flagged ones
  unsigned char flag[kBlock];
  for (int64_t b0 = i0; b0 < i1; b0 += kBlock) {
    const int64_t b1 = b0 + kBlock < i1 ? b0 + kBlock : i1;
#pragma omp simd
    for (int64_t i = b0; i < b1; ++i) {
      float mx, my, mz, p;
      bool bad;
      sample_host<METHOD, PRECISE>(h.wx[i], h.wy[i], h.wz[i], h.ax[i], ay[i], h.u1[i], h.u2[i], mx, my, mz, p,
                                   bad);
      h.mx[i] = mx;
      h.my[i] = my;
      h.mz[i] = mz;
      if constexpr (PDF) h.pdf[i] = p;
      if constexpr (PRECISE) flag[i - b0] = bad;
    }
    if constexpr (PRECISE) {
      for (int64_t i = b0; i < b1; ++i) {
        if (!flag[i - b0]) continue;
        float mx, my, mz, p;
        sample_host_double<METHOD == VNDF_METHOD_SPHERICAL_CAP_EXTENDED>(h.wx[i], h.wy[i], h.wz[i], h.ax[i], ay[i],
                                                                        h.u1[i], h.u2[i], mx, my, mz, p);
        h.mx[i] = mx;
        h.my[i] = my;
        h.mz[i] = mz;
        if constexpr (PDF) h.pdf[i] = p;
      }
    }
  }
}

template <int METHOD>
void run_method(const HostArgs& h, bool pdf, bool precise, int64_t i0, int64_t i1) {
  if (precise) {
    pdf ? run_range<METHOD, true, true>(h, i0, i1) : run_range<METHOD, false, true>(h, i0, i1);
  } else {
    pdf ? run_range<METHOD, true, false>(h, i0, i1) : run_range<METHOD, false, false>(h, i0, i1);
  }
}

// Persistent host worker threads.  Starting a thread per call and joining it cost about as much as the
// sampling itself at 2^20 samples on 16 cores, so the workers are created once and wait on a condition
// variable between calls.  A call publishes a job (a task function, its context and a task count);
// workers and the calling thread take task indices from the job's own counter until none is left,
// and the caller returns once every task has finished.  Each job is a separate object, so a worker that
// wakes late can only find an exhausted job.  Calls from several host threads are served one at a time.
// After fork() the child starts a new pool on first use (the parent's workers do not exist there).
struct Job {
  void (*fn)(void*, int);
  void* ctx;
  int tasks;
  std::atomic<int> next{0};
  std::atomic<int> left{0};
  std::mutex m;
  std::condition_variable done;
};

class WorkerPool {
 public:
  explicit WorkerPool(int workers) {
    for (int i = 0; i < workers; ++i) std::thread([this] { loop(); }).detach();
  }

  void run(int tasks, void (*fn)(void*, int), void* ctx) {
    std::lock_guard<std::mutex> serial(run_mutex_);
    auto job = std::make_shared<Job>();
    job->fn = fn;
    job->ctx = ctx;
    job->tasks = tasks;
    job->left.store(tasks);
    {
      std::lock_guard<std::mutex> lk(m_);
      job_ = job;
      ++gen_;
    }
    cv_.notify_all();
    work(*job);
    {
      std::unique_lock<std::mutex> lk(job->m);
      job->done.wait(lk, [&] { return job->left.load() == 0; });
    }
    std::lock_guard<std::mutex> lk(m_);
    if (job_ == job) job_.reset();
  }

 private:
  static void work(Job& j) {
    for (int k; (k = j.next.fetch_add(1)) < j.tasks;) {
      j.fn(j.ctx, k);
      if (j.left.fetch_sub(1) == 1) {
        std::lock_guard<std::mutex> lk(j.m);
        j.done.notify_all();
      }
    }
  }

  void loop() {
    uint64_t seen = 0;
    for (;;) {
      std::shared_ptr<Job> job;
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        job = job_;
      }
      if (job) work(*job);
    }
  }

  std::mutex run_mutex_, m_;
  std::condition_variable cv_;
  std::shared_ptr<Job> job_;
  uint64_t gen_ = 0;
};

std::atomic<WorkerPool*> g_pool{nullptr};
std::mutex g_pool_mutex;

void forget_pool_in_child() { g_pool.store(nullptr); }  // the workers were not copied by fork

WorkerPool& pool() {
  WorkerPool* p = g_pool.load();
  if (p) return *p;
  std::lock_guard<std::mutex> lk(g_pool_mutex);
  p = g_pool.load();
  if (!p) {
    static std::once_flag atfork;
    std::call_once(atfork, [] { pthread_atfork(nullptr, nullptr, forget_pool_in_child); });
    const int hw = static_cast<int>(std::thread::hardware_concurrency());
    p = new WorkerPool(hw > 1 ? hw - 1 : 1);  // lives until the process exits
    g_pool.store(p);
  }
  return *p;
}

}  // namespace

extern "C" int vndf_cpu_sample(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                               const float* alpha_x, const float* alpha_y, const float* u1, const float* u2,
                               int method, int precise, float* wm_x, float* wm_y, float* wm_z, float* pdf,
                               int threads) {
  if (n < 0 || n >= (int64_t(1) << 62)) return VNDF_ERR_SIZE;
  if (method != VNDF_METHOD_SPHERICAL_CAP && method != VNDF_METHOD_POLAR_DISK &&
      method != VNDF_METHOD_SPHERICAL_CAP_EXTENDED)
    return VNDF_ERR_METHOD;
  if (n == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !alpha_x || !u1 || !u2 || !wm_x || !wm_y || !wm_z) return VNDF_ERR_NULL;
  {  // outputs must not overlap the inputs or each other (exact equality is what can be checked)
    const void* outs[] = {wm_x, wm_y, wm_z, pdf};
    const void* ins[] = {wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2};
    for (int o = 0; o < 4; ++o) {
      if (outs[o] == nullptr) continue;
      for (int p = 0; p < o; ++p)
        if (outs[p] == outs[o]) return VNDF_ERR_ARG;
      for (const void* i : ins)
        if (i == outs[o]) return VNDF_ERR_ARG;
    }
  }
  const HostArgs h{wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wm_x, wm_y, wm_z, pdf};
  const bool want_pdf = pdf != nullptr, strict = precise != 0;
  auto body = [&](int64_t i0, int64_t i1) {
    if (method == VNDF_METHOD_SPHERICAL_CAP)
      run_method<VNDF_METHOD_SPHERICAL_CAP>(h, want_pdf, strict, i0, i1);
    else if (method == VNDF_METHOD_SPHERICAL_CAP_EXTENDED)
      run_method<VNDF_METHOD_SPHERICAL_CAP_EXTENDED>(h, want_pdf, strict, i0, i1);
    else
      run_method<VNDF_METHOD_POLAR_DISK>(h, want_pdf, false, i0, i1);  // the prior sampler has no such path
  };
  int t = threads > 0 ? threads : static_cast<int>(std::thread::hardware_concurrency());
  if (t < 1) t = 1;
  if (int64_t(t) > n / 4096) t = static_cast<int>(n / 4096 > 0 ? n / 4096 : 1);
  if (t == 1) {
    body(0, n);
    return VNDF_OK;
  }
  // t tasks of consecutive samples, so at most t threads work at once
  struct Ctx {
    decltype(body)* body;
    int64_t chunk, n;
  } ctx{&body, ((n + t - 1) / t + 15) / 16 * 16, n};
  pool().run(t, [](void* c, int k) {
    const Ctx& x = *static_cast<const Ctx*>(c);
    const int64_t i0 = int64_t(k) * x.chunk, i1 = i0 + x.chunk < x.n ? i0 + x.chunk : x.n;
    if (i0 < i1) (*x.body)(i0, i1);
  }, &ctx);
  return VNDF_OK;
}
