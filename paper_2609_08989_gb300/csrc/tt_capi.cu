// tt_capi.cu -- host side of the C ABI declared in include/tartarus.h.
//
// Validates the caller's structs, resolves per-image constants (event radii,
// ISCO, Page-Thorne roots, the observer's tetrad), zeroes a work-queue counter
// from a per-device ring on the caller's stream and enqueues the persistent
// kernel with the image descriptors as kernel parameters.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tartarus.h"
#include "tt_internal.h"

struct tt_table {
    double* d_coef;      // device patch coefficients, kTableCoef per cell
    float2* d_coef_df;   // the same as double-float pairs (hi, lo)
    int nr, nth;
    double r_min, r_max;
    int device;
};

namespace {

std::atomic<long long> g_launches{0};

bool is_finite(double x) { return std::isfinite(x); }

double kerr_rplus(double M, double a) { return M + std::sqrt(M * M - a * a); }

// the nearest double-float: hi = the float nearest v, lo = the float nearest v - hi
float2 split_df(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// Prograde ISCO, Bardeen, Press & Teukolsky (1972), a >= 0.
double kerr_isco(double M, double a) {
    const double s = a / M;
    const double z1 = 1.0 + std::cbrt(1.0 - s * s) * (std::cbrt(1.0 + s) + std::cbrt(1.0 - s));
    const double z2 = std::sqrt(3.0 * s * s + z1 * z1);
    return M * (3.0 + z2 - std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2)));
}

int check_metric(const tt_metric* m) {
    if (!m) return TT_EINVAL;
    if (m->kind != TT_METRIC_KERR && m->kind != TT_METRIC_TABLE) return TT_EINVAL;
    if (!is_finite(m->M) || !(m->M > 0.0) || !is_finite(m->a)) return TT_EINVAL;
    if (m->kind == TT_METRIC_KERR && !(std::fabs(m->a) < m->M)) return TT_EINVAL;
    if (m->kind == TT_METRIC_TABLE) {
        if (!m->table || !m->table->d_coef) return TT_EINVAL;
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev != m->table->device) return TT_EINVAL;
        if (!(std::fabs(m->a) <= m->M)) return TT_EINVAL;
    }
    return TT_OK;
}

int check_solver(const tt_solver* s) {
    if (!s) return TT_EINVAL;
    if (s->method < TT_DP54 || s->method > TT_VERLET) return TT_EINVAL;
    if (s->precision != TT_FP64 && s->precision != TT_MIXED && s->precision != TT_MIXED_PAIR &&
        s->precision != TT_DOUBLE_FLOAT && s->precision != TT_MIXED_SPLIT)
        return TT_EINVAL;
    if (s->method != TT_DP54 && s->precision != TT_FP64) return TT_EUNSUPPORTED;
    if (!is_finite(s->rtol) || !is_finite(s->atol) || !(s->rtol > 0.0) || !(s->atol > 0.0)) return TT_EINVAL;
    if (!is_finite(s->h0) || !is_finite(s->h_min)) return TT_EINVAL;
    if (s->method == TT_VERLET && !(s->h0 > 0.0)) return TT_EINVAL;     // Verlet's fixed step
    if (s->max_steps < 1) return TT_EINVAL;
    if (!is_finite(s->horizon_eps) || s->horizon_eps < 0.0) return TT_EINVAL;
    if (!is_finite(s->escape_factor) || !(s->escape_factor > 1.0)) return TT_EINVAL;
    if (s->refine != TT_REFINE_HENON && s->refine != TT_REFINE_HERMITE && s->refine != TT_REFINE_HENON64)
        return TT_EINVAL;
    if (!is_finite(s->fp64_radius_factor) || !is_finite(s->fp64_pole_sin)) return TT_EINVAL;
    if (!is_finite(s->critical_band) || !is_finite(s->critical_rtol) || s->critical_rtol < 0.0) return TT_EINVAL;
    return TT_OK;
}

bool mixed_precision(int p) { return p == TT_MIXED || p == TT_MIXED_PAIR || p == TT_MIXED_SPLIT; }

int check_outputs(const tt_outputs* o) {
    if (!o) return TT_EINVAL;
    if (!o->code || !o->n_cross || !o->r_cross || !o->g || !o->I_cross || !o->intensity || !o->h_max ||
        !o->steps || !o->rejects)
        return TT_EINVAL;
    return TT_OK;
}

#ifdef TT_BOUNDS_CHECK
// The bounds-checking build's fault counter: a file-scope device variable (no
// allocation), its address looked up once per device.
static __device__ unsigned long long tt_fault_count;
unsigned long long* g_fault_addr[64] = {};
std::mutex g_fault_mu;

unsigned long long* fault_counter() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (!g_fault_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, tt_fault_count) != cudaSuccess) return nullptr;
        g_fault_addr[dev] = static_cast<unsigned long long*>(p);
    }
    return g_fault_addr[dev];
}
#endif

// Resolve one image into a kernel descriptor.
int make_desc(const tt_metric* m, const tt_observer* obs, const tt_camera* cam, const tt_solver* sol,
              const tt_disk* disk, const tt_outputs* out, tt::ImageDesc* d) {
    int rc = check_metric(m);
    if (rc) return rc;
    if (!obs || !cam || !disk) return TT_EINVAL;
    if (!is_finite(obs->r_obs) || !(obs->r_obs > 0.0)) return TT_EINVAL;
    if (!is_finite(obs->theta_obs) || !(obs->theta_obs > 0.0) || !(obs->theta_obs < M_PI)) return TT_EINVAL;
    if (cam->nx < 1 || cam->ny < 1) return TT_EINVAL;
    if (!is_finite(cam->alpha_min) || !is_finite(cam->alpha_max) || !is_finite(cam->beta_min) || !is_finite(cam->beta_max))
        return TT_EINVAL;
    const long long npix = (long long)cam->nx * (long long)cam->ny;
    if (cam->pix_begin < 0 || cam->pix_begin > npix) return TT_EINVAL;
    long long count = cam->pix_count > 0 ? cam->pix_count : npix - cam->pix_begin;
    if (cam->pix_begin + count > npix) return TT_EINVAL;
    if (count > 0 && check_outputs(out)) return TT_EINVAL;
    if (disk->enabled) {
        if (!is_finite(disk->r_in) || !is_finite(disk->r_out) || !is_finite(disk->mdot)) return TT_EINVAL;
        if (!(disk->r_out > 0.0)) return TT_EINVAL;
        if (disk->max_crossings < 0 || disk->max_crossings > TT_MAX_CROSSINGS) return TT_EINVAL;
        if (m->a < 0.0) return TT_EINVAL;          // the prograde Keplerian disk needs a >= 0
    }
    std::memset(d, 0, sizeof *d);
    d->nx = cam->nx;
    d->ny = cam->ny;
    d->pix_begin = cam->pix_begin;
    d->pix_count = count;
    d->alpha_min = cam->alpha_min;
    d->dalpha = (cam->alpha_max - cam->alpha_min) / (double)cam->nx;
    d->beta_min = cam->beta_min;
    d->dbeta = (cam->beta_max - cam->beta_min) / (double)cam->ny;
    d->r_obs = obs->r_obs;
    d->theta_obs = obs->theta_obs;
    d->kind = m->kind;
    d->M = m->M;
    d->a = m->a;
    double r_h;
    if (m->kind == TT_METRIC_TABLE && sol->precision != TT_FP64 && sol->precision != TT_DOUBLE_FLOAT)
        return TT_EUNSUPPORTED;
    if (m->kind == TT_METRIC_TABLE) {
        const tt_table* t = m->table;
        d->table = t->d_coef;
        d->table_df = t->d_coef_df;
        d->nr = t->nr;
        d->nth = t->nth;
        d->u0 = std::log(t->r_min);
        d->du = (std::log(t->r_max) - d->u0) / (double)(t->nr - 1);
        d->dth = M_PI / (double)(t->nth - 1);
        d->u0_df = split_df(d->u0);
        d->idu_df = split_df(1.0 / d->du);
        d->idth_df = split_df(1.0 / d->dth);
        r_h = t->r_min;
    } else {
        r_h = kerr_rplus(m->M, m->a);
        d->r_plus = r_h;
        d->r_minus = m->M - std::sqrt(m->M * m->M - m->a * m->a);
        // the observer's metric and ZAMO tetrad are the same for every pixel
        const double M = m->M, a = m->a, r = obs->r_obs;
        const double s = std::sin(obs->theta_obs), c = std::cos(obs->theta_obs), s2 = s * s;
        const double Sig = r * r + a * a * c * c, Del = r * r - 2.0 * M * r + a * a;
        const double g[5] = {-(1.0 - 2.0 * M * r / Sig), -2.0 * M * a * r * s2 / Sig, Sig / Del, Sig,
                             (r * r + a * a + 2.0 * M * a * a * r * s2 / Sig) * s2};
        const double omega = -g[1] / g[4];
        const double N = std::sqrt(-g[0] + omega * omega * g[4]);
        for (int i = 0; i < 5; ++i) d->obs_g[i] = g[i];
        d->obs_omN = omega / N;
        d->obs_iN = 1.0 / N;
        d->obs_ir = 1.0 / std::sqrt(g[2]);
        d->obs_ith = 1.0 / std::sqrt(g[3]);
        d->obs_iph = 1.0 / std::sqrt(g[4]);
        d->obs_ready = 1;
    }
    d->r_capture = r_h * (1.0 + sol->horizon_eps);
    d->r_escape = sol->escape_factor * obs->r_obs;
    // mixed paths: steps starting below r_fp64 run in double-float (TT_MIXED_SPLIT:
    // FP64) (factor 0 -> 1.5, negative -> never), and those within
    // asin(fp64_pole_sin) of the axis (0 or negative -> never: the FP32 stages
    // take theta relative to the nearest axis crossing, which keeps |H| <= 1e-6
    // on every escaped ray of the benchmark image and of the 64-image batch
    // without a polar zone).  Double-float path on a table: the same zones run in
    // FP64, with the radius factor 2 by default.
    const bool df_table = m->kind == TT_METRIC_TABLE && sol->precision == TT_DOUBLE_FLOAT;
    const double pole_sin = sol->fp64_pole_sin != 0.0 ? sol->fp64_pole_sin : -1.0;
    const double radius_default = df_table ? 2.0 : 1.5;
    d->r_fp64 = sol->fp64_radius_factor < 0.0
                    ? 0.0
                    : (sol->fp64_radius_factor > 0.0 ? sol->fp64_radius_factor : radius_default) * r_h;
    d->th_pole = pole_sin < 0.0 ? 0.0 : std::asin(std::min(1.0, pole_sin));
    d->disk = disk->enabled ? 1 : 0;
    d->max_cross = disk->enabled ? disk->max_crossings : 0;
    d->doppler = disk->doppler ? 1 : 0;
    d->mdot = disk->mdot;
    d->r_out = disk->r_out;
    d->sqrtM = std::sqrt(m->M);
    if (disk->enabled) {
        const double risco = kerr_isco(m->M, m->a);
        d->r_in = disk->r_in > 0.0 ? disk->r_in : risco;
        // Page-Thorne constants (paper Sec. 2.3): x = sqrt(r/M), roots of x^3 - 3x + 2a.
        const double as = m->a / m->M;
        d->fa = as;
        d->fx0 = std::sqrt(risco / m->M);
        const double ac = std::acos(as);
        const double xr[3] = {2.0 * std::cos((ac - M_PI) / 3.0), 2.0 * std::cos((ac + M_PI) / 3.0),
                              -2.0 * std::cos(ac / 3.0)};
        for (int i = 0; i < 3; ++i) {
            d->fxr[i] = xr[i];
            if (xr[i] == 0.0) {                  // a = 0: the vanishing term of the limit
                d->fcoef[i] = 0.0;
                d->flog0[i] = 0.0;
                continue;
            }
            double prod = 1.0;
            for (int j = 0; j < 3; ++j)
                if (j != i) prod *= (xr[i] - xr[j]);
            d->fcoef[i] = 3.0 * (xr[i] - as) * (xr[i] - as) / (xr[i] * prod);
            d->flog0[i] = std::log(d->fx0 - xr[i]);
        }
        d->flux_scale = disk->mdot / (m->M * m->M);
    }
    if (count > 0) {
        d->code = out->code;
        d->n_cross = out->n_cross;
        d->r_cross = out->r_cross;
        d->g = out->g;
        d->I_cross = out->I_cross;
        d->intensity = out->intensity;
        d->h_max = out->h_max;
        d->steps = out->steps;
        d->rejects = out->rejects;
    }
    return TT_OK;
}

tt::SolverDesc make_solver(const tt_solver* s) {
    tt::SolverDesc sd;
    sd.rtol = s->rtol;
    sd.atol = s->atol;
    sd.h0 = s->h0;
    sd.h_min = s->h_min;
    sd.max_steps = s->max_steps;
    sd.refine = s->refine;
    sd.precision = s->precision;
    sd.method = s->method;
    // near-critical rays in double-float: mixed paths only (default band 0.15 M,
    // none on the prescribed split), at the FP64 path's tolerance by default
    sd.crit_band = 0.0;
    sd.crit_rtol = sd.crit_atol = 0.0;
#ifdef TT_BOUNDS_CHECK
    sd.faults = fault_counter();
#else
    sd.faults = nullptr;
#endif
    if (mixed_precision(s->precision)) {
        const double band_default = s->precision == TT_MIXED_SPLIT ? -1.0 : 0.15;
        const double band = s->critical_band != 0.0 ? s->critical_band : band_default;
        sd.crit_band = band > 0.0 ? band : 0.0;
        sd.crit_rtol = sd.crit_atol = s->critical_rtol > 0.0 ? s->critical_rtol : 1e-10;
    }
    return sd;
}

tt::LaunchShape make_shape(const tt_tune* t) {
    tt::LaunchShape s{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};       // zeros: the kernel's defaults
    if (t) {
        if (t->block > 0) s.block = t->block;
        if (t->reg_variant > 0) s.reg_variant = t->reg_variant;
        if (t->refill > 0) s.refill = t->refill;
        if (t->blocks_per_sm > 0) s.blocks_per_sm = t->blocks_per_sm;
        if (t->crossing_batch > 0) s.crossing_batch = t->crossing_batch;
        if (t->fp64_batch > 0) s.fp64_batch = t->fp64_batch;
        if (t->monitor_period > 0) s.monitor_period = t->monitor_period;
        if (t->fp64_wait > 0) s.fp64_wait = t->fp64_wait;
        if (t->crit_stride > 0) s.crit_stride = t->crit_stride;
        if (t->crit_refill > 0) s.crit_refill = t->crit_refill;
    }
    return s;
}

int check_shape(const tt_tune* t) {
    if (!t) return TT_OK;
    if (t->block != 0 && t->block != 128 && t->block != 256 && t->block != 384) return TT_EUNSUPPORTED;
    // built variants: 128, 256 or 384 threads (FP64 Dormand-Prince, closed-form Kerr),
    // 128 or 256 (the other FP64 integrators; 384 runs as 256), 128 (FP64 tables),
    // 256 (mixed paths; 384 runs as 256, 128 is refused at launch)
    if (t->reg_variant < 0 || t->reg_variant > 2) return TT_EUNSUPPORTED;
    if (t->refill < 0 || t->refill > 32) return TT_EINVAL;
    if (t->blocks_per_sm < 0) return TT_EINVAL;
    if (t->crossing_batch < 0 || t->crossing_batch > 32) return TT_EINVAL;
    if (t->fp64_batch < 0 || t->fp64_batch > 32) return TT_EINVAL;
    if (t->monitor_period < 0 || t->fp64_wait < 0) return TT_EINVAL;
    if (t->crit_stride < 0 || t->crit_refill < 0 || t->crit_refill > 32) return TT_EINVAL;
    return TT_OK;
}

// The kernels of the integrators other than Dormand-Prince, and the
// double-float kernels, take one metric kind per launch: a batch with both
// closed-form Kerr and tabulated images is refused for them.
int check_kinds(const tt_image* images, int n, const tt_solver* s) {
    if (s->method == TT_DP54 && s->precision != TT_DOUBLE_FLOAT) return TT_OK;
    bool kerr = false, table = false;
    for (int i = 0; i < n; ++i) {
        if (images[i].metric.kind == TT_METRIC_TABLE) table = true;
        else kerr = true;
    }
    return (kerr && table) ? TT_EUNSUPPORTED : TT_OK;
}

// Work-queue counters: one small device array per device, allocated on the
// first call on that device and kept until the process exits.  Each call takes
// the next slot (round robin) and zeroes it on its stream before the launch,
// so up to kQueueSlots calls may be in flight on one device at once.
constexpr int kQueueSlots = 1024;
constexpr int kMaxDevices = 64;
std::mutex g_queue_mu;
unsigned long long* g_queue[kMaxDevices] = {};
std::atomic<unsigned> g_queue_next[kMaxDevices];

unsigned long long* queue_slot() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    {
        std::lock_guard<std::mutex> lk(g_queue_mu);
        if (!g_queue[dev]) {
            unsigned long long* p = nullptr;
            if (cudaMalloc((void**)&p, kQueueSlots * 32 * sizeof(unsigned long long)) != cudaSuccess) return nullptr;
            g_queue[dev] = p;
        }
    }
    const unsigned k = g_queue_next[dev].fetch_add(1) % kQueueSlots;
    return g_queue[dev] + (size_t)k * 32;           // one 256-byte line per slot
}

// The device-side output block of tartarus_trace_host comes from the device's
// default stream-ordered pool; keep freed blocks in the pool instead of
// returning them to the CUDA runtime at every synchronisation.
void keep_pool_memory() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
    static std::atomic<bool> done[kMaxDevices];
    if (done[dev].exchange(true)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
}

// Zero a queue slot and launch; batches larger than one launch's capacity are
// split into consecutive launches on the same stream.
int enqueue(const std::vector<tt::ImageDesc>& descs, const tt_solver* sol, const tt_tune* tune,
            cudaStream_t st) {
    const tt::SolverDesc sd = make_solver(sol);
    const tt::LaunchShape shape = make_shape(tune);
    for (size_t first = 0; first < descs.size(); first += tt::kMaxImagesPerLaunch) {
        const size_t n = std::min(descs.size() - first, (size_t)tt::kMaxImagesPerLaunch);
        tt::ImageDesc ds[tt::kMaxImagesPerLaunch];
        long long total = 0;
        int n_table = 0;
        for (size_t i = 0; i < n; ++i) {
            ds[i] = descs[first + i];
            ds[i].ray_begin = total;
            total += ds[i].pix_count;
            n_table += ds[i].kind == TT_METRIC_TABLE;
        }
        if (total == 0) continue;
        // 0: closed-form Kerr only, 1: tables only, 2: both kinds (dispatch per ray)
        const int metric_mode = n_table == 0 ? 0 : (n_table == (int)n ? 1 : 2);
        unsigned long long* q = queue_slot();
        if (!q) return TT_ENOMEM;
        cudaError_t e = cudaMemsetAsync(q, 0, 2 * sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = tt::launch_trace(ds, (int)n, total, metric_mode, sd, shape, q, st);
        if (e != cudaSuccess) return TT_ECUDA;
        g_launches.fetch_add(1);
    }
    return TT_OK;
}

// ---------------------------------------------------------------------------
// Fixed device scratch for tartarus_trace_batch_noalloc.
//
// The tracer's only scratch is one 64-bit work-queue counter per launch (a
// launch covers up to kMaxImagesPerLaunch images).  For callers that may not
// allocate, those counters live in this file-scope array instead of the
// lazily allocated ring above: kNoAllocSlots counters, one 256-byte line each
// (4 KiB in all), present on every device that loads the library until the
// process exits.  A call needs ceil(n / 64) counters, so it takes at most
// kNoAllocSlots * 64 = 1024 images.  Host code must not pass the symbol
// itself to a kernel (on the host it names a stand-in, not device memory):
// its device address is looked up once per device and cached.
// ---------------------------------------------------------------------------
constexpr int kNoAllocSlots = 16;
constexpr int kNoAllocMaxImages = kNoAllocSlots * tt::kMaxImagesPerLaunch;
static __device__ __align__(256) unsigned long long tt_noalloc_queue[kNoAllocSlots * 32];
unsigned long long* g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of the fixed scratch on the current device (looked up on the
// first call on that device, with that device current).
int noalloc_scratch(unsigned long long** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TT_ECUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, tt_noalloc_queue) != cudaSuccess || !p) return TT_ECUDA;
        g_noalloc_addr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_noalloc_addr[dev];
    return TT_OK;
}

}  // namespace

extern "C" {

int tartarus_trace_batch_noalloc(const tt_image* images, int n, const tt_solver* solver, const tt_tune* tune,
                                 int* status, void* cuda_stream) {
    if (n < 0 || (n > 0 && !images)) return TT_EINVAL;
    if (n > kNoAllocMaxImages) return TT_EINVAL;           // more counters than the fixed scratch holds
    int rc = check_solver(solver);
    if (rc) return rc;
    rc = check_shape(tune);
    if (rc) return rc;
    rc = check_kinds(images, n, solver);
    if (rc) return rc;
    unsigned long long* scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const tt::SolverDesc sd = make_solver(solver);
    const tt::LaunchShape shape = make_shape(tune);
    int worst = TT_OK;
    // every image is validated (and its status written) before the first launch
    for (int i = 0; i < n; ++i) {
        tt::ImageDesc d;
        const tt_image& im = images[i];
        const int r = make_desc(&im.metric, &im.obs, &im.cam, solver, &im.disk, &im.out, &d);
        if (status) status[i] = r;
        if (r) worst = r;
    }
    int slot = 0;
    tt::ImageDesc ds[tt::kMaxImagesPerLaunch];
    int nd = 0;
    long long total = 0;
    int n_table = 0;
    // then the valid ones are launched chunk by chunk (fixed-size host arrays, no heap)
    for (int i = 0; i <= n; ++i) {
        if (i < n) {
            tt::ImageDesc d;
            const tt_image& im = images[i];
            if (make_desc(&im.metric, &im.obs, &im.cam, solver, &im.disk, &im.out, &d)) continue;
            if (d.pix_count == 0) continue;
            d.ray_begin = total;
            total += d.pix_count;
            n_table += d.kind == TT_METRIC_TABLE;
            ds[nd++] = d;
        }
        if ((nd == tt::kMaxImagesPerLaunch || i == n) && nd > 0) {
            unsigned long long* q = scratch + (size_t)slot * 32;
            ++slot;
            const int metric_mode = n_table == 0 ? 0 : (n_table == nd ? 1 : 2);
            // the array keeps the previous call's counts: zero this launch's counters first
            cudaError_t e = cudaMemsetAsync(q, 0, 2 * sizeof(unsigned long long), st);
            if (e == cudaSuccess) e = tt::launch_trace(ds, nd, total, metric_mode, sd, shape, q, st);
            if (e != cudaSuccess) return TT_ECUDA;
            g_launches.fetch_add(1);
            nd = 0;
            total = 0;
            n_table = 0;
        }
    }
    return worst;
}


int tartarus_trace(const tt_metric* metric, const tt_observer* obs, const tt_camera* cam, const tt_solver* solver,
                   const tt_disk* disk, const tt_outputs* out, const tt_tune* tune, void* cuda_stream) {
    int rc = check_solver(solver);
    if (rc) return rc;
    rc = check_shape(tune);
    if (rc) return rc;
    std::vector<tt::ImageDesc> d(1);
    rc = make_desc(metric, obs, cam, solver, disk, out, &d[0]);
    if (rc) return rc;
    return enqueue(d, solver, tune, (cudaStream_t)cuda_stream);
}

int tartarus_trace_host(const tt_metric* metric, const tt_observer* obs, const tt_camera* cam,
                        const tt_solver* solver, const tt_disk* disk, const tt_outputs* host_out,
                        const tt_tune* tune, void* cuda_stream) {
    int rc = check_solver(solver);
    if (rc) return rc;
    rc = check_shape(tune);
    if (rc) return rc;
    if (check_outputs(host_out)) return TT_EINVAL;
    if (!cam) return TT_EINVAL;
    const long long npix = (long long)cam->nx * (long long)cam->ny;
    const long long n = cam->pix_count > 0 ? cam->pix_count : npix - cam->pix_begin;
    if (cam->nx < 1 || cam->ny < 1 || n < 0) return TT_EINVAL;
    if (n == 0) return TT_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    keep_pool_memory();
    // one device block for all outputs: doubles first (8-byte aligned), then int32, then int8
    const size_t nd = (size_t)n * (3 * 3 + 2), ni = (size_t)n * 2, nb = (size_t)n * 2;
    const size_t bytes = nd * 8 + ni * 4 + nb;
    char* base = nullptr;
    if (cudaMallocAsync((void**)&base, bytes, st) != cudaSuccess) return TT_ENOMEM;
    double* dd = reinterpret_cast<double*>(base);
    int32_t* di = reinterpret_cast<int32_t*>(base + nd * 8);
    int8_t* db = reinterpret_cast<int8_t*>(base + nd * 8 + ni * 4);
    tt_outputs dev;
    dev.r_cross = dd;
    dev.g = dd + 3 * n;
    dev.I_cross = dd + 6 * n;
    dev.intensity = dd + 9 * n;
    dev.h_max = dd + 10 * n;
    dev.steps = di;
    dev.rejects = di + n;
    dev.code = db;
    dev.n_cross = db + n;
    rc = tartarus_trace(metric, obs, cam, solver, disk, &dev, tune, cuda_stream);
    if (rc == TT_OK) {
        cudaError_t e = cudaSuccess;
        auto cp = [&](void* dst, const void* src, size_t b) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, st);
        };
        cp(host_out->r_cross, dev.r_cross, 3 * n * 8);
        cp(host_out->g, dev.g, 3 * n * 8);
        cp(host_out->I_cross, dev.I_cross, 3 * n * 8);
        cp(host_out->intensity, dev.intensity, n * 8);
        cp(host_out->h_max, dev.h_max, n * 8);
        cp(host_out->steps, dev.steps, n * 4);
        cp(host_out->rejects, dev.rejects, n * 4);
        cp(host_out->code, dev.code, n);
        cp(host_out->n_cross, dev.n_cross, n);
        if (e != cudaSuccess) rc = TT_ECUDA;
    }
    cudaFreeAsync(base, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == TT_OK) rc = TT_ECUDA;
    return rc;
}

int tartarus_trace_batch(const tt_image* images, int n, const tt_solver* solver, const tt_tune* tune, int* status,
                         void* cuda_stream) {
    if (n < 0 || (n > 0 && !images)) return TT_EINVAL;
    int rc = check_solver(solver);
    if (rc) return rc;
    rc = check_shape(tune);
    if (rc) return rc;
    rc = check_kinds(images, n, solver);
    if (rc) return rc;
    std::vector<tt::ImageDesc> descs;
    descs.reserve(n);
    int worst = TT_OK;
    for (int i = 0; i < n; ++i) {
        tt::ImageDesc d;
        const tt_image& im = images[i];
        int r = make_desc(&im.metric, &im.obs, &im.cam, solver, &im.disk, &im.out, &d);
        if (status) status[i] = r;
        if (r) {
            worst = r;
            continue;
        }
        if (d.pix_count > 0) descs.push_back(d);
    }
    if (!descs.empty()) {
        int e = enqueue(descs, solver, tune, (cudaStream_t)cuda_stream);
        if (e) return e;
    }
    return worst;
}

// The per-cell patch coefficients of a node table (validated), host only.
static int table_coefficients(const double* host_nodes, int nr, int nth, double r_min, double r_max,
                              std::vector<double>& cf) {
    if (!host_nodes || nr < 2 || nth < 2) return TT_EINVAL;
    if (!is_finite(r_min) || !is_finite(r_max) || !(r_min > 0.0) || !(r_max > r_min)) return TT_EINVAL;
    const size_t n = (size_t)nr * (size_t)nth * tt::kTableNF;
    std::vector<double> loc(n);
    const double u0 = std::log(r_min);
    const double du = (std::log(r_max) - u0) / (double)(nr - 1);
    const double dth = M_PI / (double)(nth - 1);
    for (int j = 0; j < nth; ++j) {
        for (int k = 0; k < nr; ++k) {
            const double rk = std::exp(u0 + (double)k * du);
            const double* src = host_nodes + ((size_t)j * nr + k) * tt::kTableNF;
            double* dst = loc.data() + ((size_t)j * nr + k) * tt::kTableNF;
            for (int f = 0; f < 5; ++f) {
                const double F = src[4 * f], Fr = src[4 * f + 1], Ft = src[4 * f + 2], Frt = src[4 * f + 3];
                if (!is_finite(F) || !is_finite(Fr) || !is_finite(Ft) || !is_finite(Frt)) return TT_EINVAL;
                dst[4 * f] = F;
                dst[4 * f + 1] = rk * Fr * du;           // slope in the unit-cell u coordinate
                dst[4 * f + 2] = Ft * dth;               // slope in the unit-cell theta coordinate
                dst[4 * f + 3] = rk * Frt * du * dth;    // twist
            }
        }
    }
    // Per cell and field, the bicubic Hermite patch in the monomial basis,
    // v(t, w) = sum_ij c_ij t^i w^j: C = Hm^T G Hm, where G[m][n] is the
    // coefficient of h_m(t) h_n(w) (m = 2 cu + u-slope, n = 2 ct + theta-slope
    // for the corner (cu, ct)) and row m of Hm the power coefficients of h_m:
    // h0 = 1 - 3t^2 + 2t^3, h1 = t - 2t^2 + t^3, h2 = 3t^2 - 2t^3, h3 = t^3 - t^2.
    // The same polynomial as the Hermite form; it evaluates by Horner's rule
    // with half the multiply-adds and no basis functions.
    static const double Hm[4][4] = {{1, 0, -3, 2}, {0, 1, -2, 1}, {0, 0, 3, -2}, {0, 0, -1, 1}};
    const size_t ncoef = (size_t)(nr - 1) * (size_t)(nth - 1) * tt::kTableCoef;
    cf.assign(ncoef, 0.0);
    for (int j = 0; j + 1 < nth; ++j) {
        for (int k = 0; k + 1 < nr; ++k) {
            double* dst = cf.data() + ((size_t)j * (nr - 1) + k) * tt::kTableCoef;
            for (int f = 0; f < 5; ++f) {
                double G[4][4];
                for (int ct = 0; ct < 2; ++ct) {
                    for (int cu = 0; cu < 2; ++cu) {
                        const double* nd = loc.data() + ((size_t)(j + ct) * nr + (k + cu)) * tt::kTableNF + 4 * f;
                        G[2 * cu][2 * ct] = nd[0];
                        G[2 * cu + 1][2 * ct] = nd[1];
                        G[2 * cu][2 * ct + 1] = nd[2];
                        G[2 * cu + 1][2 * ct + 1] = nd[3];
                    }
                }
                double GH[4][4];          // G Hm
                for (int m = 0; m < 4; ++m)
                    for (int q = 0; q < 4; ++q) {
                        double acc = 0.0;
                        for (int n2 = 0; n2 < 4; ++n2) acc += G[m][n2] * Hm[n2][q];
                        GH[m][q] = acc;
                    }
                for (int i = 0; i < 4; ++i)
                    for (int q = 0; q < 4; ++q) {
                        double acc = 0.0;
                        for (int m = 0; m < 4; ++m) acc += Hm[m][i] * GH[m][q];
                        dst[16 * f + 4 * i + q] = acc;
                    }
            }
        }
    }
    return TT_OK;
}

int tartarus_table_coefficients(const double* host_nodes, int nr, int nth, double r_min, double r_max,
                                double* out) {
    if (!out) return TT_EINVAL;
    std::vector<double> cf;
    const int rc = table_coefficients(host_nodes, nr, nth, r_min, r_max, cf);
    if (rc) return rc;
    std::copy(cf.begin(), cf.end(), out);
    return TT_OK;
}

int tartarus_table_create(const double* host_nodes, int nr, int nth, double r_min, double r_max, tt_table** out) {
    if (!out) return TT_EINVAL;
    *out = nullptr;
    std::vector<double> cf;
    const int rc = table_coefficients(host_nodes, nr, nth, r_min, r_max, cf);
    if (rc) return rc;
    const size_t ncoef = cf.size();
    // the double-float copy
    std::vector<float2> cdf(ncoef);
    for (size_t i = 0; i < ncoef; ++i) cdf[i] = split_df(cf[i]);
    tt_table* t = new (std::nothrow) tt_table;
    if (!t) return TT_ENOMEM;
    t->d_coef = nullptr;
    t->d_coef_df = nullptr;
    cudaGetDevice(&t->device);
    if (cudaMalloc((void**)&t->d_coef, ncoef * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&t->d_coef_df, ncoef * sizeof(float2)) != cudaSuccess) {
        cudaFree(t->d_coef);
        delete t;
        return TT_ENOMEM;
    }
    if (cudaMemcpy(t->d_coef, cf.data(), ncoef * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_coef_df, cdf.data(), ncoef * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(t->d_coef);
        cudaFree(t->d_coef_df);
        delete t;
        return TT_ECUDA;
    }
    t->nr = nr;
    t->nth = nth;
    t->r_min = r_min;
    t->r_max = r_max;
    *out = t;
    return TT_OK;
}

int tartarus_table_destroy(tt_table* t) {
    if (!t) return TT_EINVAL;
    cudaError_t e = cudaFree(t->d_coef);
    const cudaError_t e2 = cudaFree(t->d_coef_df);
    delete t;
    return (e == cudaSuccess && e2 == cudaSuccess) ? TT_OK : TT_ECUDA;
}

const char* tartarus_error_string(int status) {
    switch (status) {
        case TT_OK: return "ok";
        case TT_EINVAL: return "invalid argument";
        case TT_ENOMEM: return "out of memory";
        case TT_ECUDA: return "CUDA runtime error";
        case TT_EUNSUPPORTED: return "unsupported variant";
        default: return "unknown status";
    }
}

long long tartarus_launch_count(void) { return g_launches.load(); }

int tartarus_debug_faults(long long* count) {
    if (!count) return TT_EINVAL;
#ifdef TT_BOUNDS_CHECK
    unsigned long long* p = fault_counter();
    if (!p) return TT_ECUDA;
    unsigned long long v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return TT_ECUDA;
    if (cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return TT_ECUDA;
    if (cudaMemset(p, 0, sizeof v) != cudaSuccess) return TT_ECUDA;
    *count = (long long)v;
    return TT_OK;
#else
    *count = 0;
    return TT_EUNSUPPORTED;
#endif
}

const char* tartarus_version(void) {
#ifdef TT_BOUNDS_CHECK
    return "tartarus-gb300 0.2 (sm_103a, bounds-checking build)";
#else
    return "tartarus-gb300 0.2 (sm_103a)";
#endif
}

}  // extern "C"
