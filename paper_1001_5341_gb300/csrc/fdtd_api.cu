// fdtd_api.cu -- the C ABI of include/fdtd.h: handle life cycle, host-side
// argument checks, device memory, the step loop and the copies in and out.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "fdtd_internal.h"

using namespace fdtd;

namespace {

constexpr double kC = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;

int note(fdtd_ctx *h, cudaError_t e) {
    if (e == cudaSuccess) return FDTD_OK;
    // FDTD_DEBUG set in the environment: the CUDA error behind a status on stderr
    static const bool debug = std::getenv("FDTD_DEBUG") != nullptr;
    if (debug) std::fprintf(stderr, "fdtd: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
    int code = (e == cudaErrorMemoryAllocation) ? FDTD_ERR_OOM : FDTD_ERR_CUDA;
    if (h && h->status == FDTD_OK) h->status = code;
    return code;
}

#define TRY(h, expr)                                  \
    do {                                              \
        int rc_ = note((h), (expr));                  \
        if (rc_ != FDTD_OK) return rc_;               \
    } while (0)

void free_dev(void *p) {
    if (p) cudaFree(p);
}

void release(fdtd_ctx *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_dev(h->fields[0]);
    free_dev(h->fields[1]);
    free_dev(h->psi_block);
    free_dev(h->epsi2);
    free_dev(h->coef_block);
    free_dev(h->d_q);
    free_dev(h->d_w);
    free_dev(h->d_ijk);
    free_dev(h->d_cxy);
    free_dev(h->d_trace);
    free_dev(h->d_partial);
    free_dev(h->d_result);
    free_dev(h->d_flags);
    vtile_release(h);
    tb2_release(h);
    for (cudaEvent_t e : h->timing.ev) cudaEventDestroy(e);
    delete h;
}

int interior_lo(const fdtd_ctx *h) { return h->boundary == FDTD_CPML ? h->P + 1 : 1; }

size_t field_bytes(const fdtd_ctx *h) { return sizeof(float) * 6 * (size_t)h->g.comp; }

}  // namespace

namespace fdtd {
Cpml cpml_view(const fdtd_ctx *h) {
    Cpml v{};
    v.P = h->P;
    v.W = h->P > 0 ? 2 * h->P + 1 : 0;
    if (h->P <= 0) return v;
    float *p = h->ecur ? h->epsi2 : h->psi_block;
    const size_t set = 2 * (h->psi_axis[0] + h->psi_axis[1] + h->psi_axis[2]);
    float *hin = h->psi_block + set * (1 + h->cur), *hout = h->psi_block + set * (1 + (h->cur ^ 1));
    size_t off = 0;
    for (int a = 0; a < 3; ++a)
        for (int t = 0; t < 2; ++t) {
            v.e[a][t] = p + off;
            v.hin[a][t] = hin + off;
            v.hout[a][t] = hout + off;
            off += h->psi_axis[a];
        }
    for (int a = 0; a < 3; ++a) {
        v.aE[a] = h->aE[a]; v.bE[a] = h->bE[a]; v.aH[a] = h->aH[a]; v.bH[a] = h->bH[a];
    }
    return v;
}

static void timed_launch(fdtd_ctx *h, cudaStream_t st, void (*fn)(const fdtd_ctx *, cudaStream_t)) {
    TimingRec &t = h->timing;
    bool rec = t.on && t.used < t.cap;
    if (rec) cudaEventRecord(t.ev[2 * t.used], st);
    fn(h, st);
    if (rec) {
        cudaEventRecord(t.ev[2 * t.used + 1], st);
        t.used++;
    }
    h->launches++;
}

// n steps of the handle's selected path, issued on `st` (the handle's own
// stream for fdtd_step; a batch's stream when the batch steps it alone).
int fdtd_step_on(fdtd_ctx *h, int n, cudaStream_t st) {
    for (int s = 0; s < n;) {
        int adv = 1;
        if (h->kernel == 2 && n - s >= 2) {
            // two steps in one pass; the detectors of both from its records
            timed_launch(h, st, [](const fdtd_ctx *c, cudaStream_t q) { launch_tb2(const_cast<fdtd_ctx *>(c), q); });
            if (h->np > 0) { launch_tb2_probes(h, st); h->launches++; }
            h->ecur ^= 1;
            adv = 2;
        } else {
            if (h->kernel == 1 || (h->kernel == 2 && h->vtile)) {
                timed_launch(h, st, [](const fdtd_ctx *c, cudaStream_t q) { launch_vtile(const_cast<fdtd_ctx *>(c), q); });
            } else {
                timed_launch(h, st, launch_update_h);
                timed_launch(h, st, launch_update_e);
            }
            if (h->boundary == FDTD_MUR1) { launch_mur(h, st); h->launches++; }
            if (h->np > 0) { launch_probes(h, st); h->launches++; }
        }
        h->cur ^= 1;
        h->steps += adv;
        s += adv;
        if (h->watch_every > 0 && h->steps / h->watch_every != (h->steps - adv) / h->watch_every) {
            launch_watch(h, st);
            h->launches++;
        }
    }
    return note(h, cudaGetLastError());
}

}  // namespace fdtd

extern "C" {

const char *fdtd_strerror(int s) {
    switch (s) {
    case FDTD_OK: return "ok";
    case FDTD_ERR_ARG: return "invalid argument";
    case FDTD_ERR_CFL: return "time step above the 3D Courant limit";
    case FDTD_ERR_OOM: return "device memory allocation failed";
    case FDTD_ERR_UNSTABLE: return "non-finite field value";
    case FDTD_ERR_CUDA: return "CUDA runtime error";
    case FDTD_ERR_TIMEOUT: return "device wait timed out";
    case FDTD_ERR_CAPACITY: return "detector trace capacity exceeded";
    default: return "unknown status";
    }
}

int fdtd_create(fdtd_t *out, int nx, int ny, int nz, double dx, double dt, double eps_r,
                int boundary, int npml, void *cuda_stream) {
    if (!out) return FDTD_ERR_ARG;
    *out = nullptr;
    if (nx < 4 || ny < 4 || nz < 4 || nx > 32000 || ny > 32000 || nz > 32000) return FDTD_ERR_ARG;
    if (!(dx > 0.0) || !(dt > 0.0) || !(eps_r >= 1.0) || !std::isfinite(dx) || !std::isfinite(eps_r))
        return FDTD_ERR_ARG;
    if (boundary != FDTD_PEC && boundary != FDTD_MUR1 && boundary != FDTD_CPML) return FDTD_ERR_ARG;
    int P = 0;
    if (boundary == FDTD_CPML) {
        if (npml < 1 || nx < 2 * npml + 4 || ny < 2 * npml + 4 || nz < 2 * npml + 4) return FDTD_ERR_ARG;
        P = npml;
    }
    const double dt_max = dx * std::sqrt(eps_r) / (kC * std::sqrt(3.0));
    if (dt > dt_max * (1.0 + 1e-12)) return FDTD_ERR_CFL;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return FDTD_ERR_CUDA;
    }
    fdtd_ctx *h = new (std::nothrow) fdtd_ctx();
    if (!h) return FDTD_ERR_OOM;
    cudaGetDevice(&h->dev);
    h->stream = (cudaStream_t)cuda_stream;
    h->boundary = boundary;
    h->P = P;
    h->dx = dx;
    h->dt = dt;
    h->eps_r = eps_r;
    h->eps = eps_r / (kMu0 * kC * kC);
    h->kE = dt / (h->eps * dx);
    h->kH = dt / (kMu0 * dx);
    const double S = kC / std::sqrt(eps_r) * dt / dx;
    h->mur_m = (S - 1.0) / (S + 1.0);
    Grid &g = h->g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.pitch = ((nx + 1) + 31) / 32 * 32;
    g.plane = (long long)(ny + 1) * g.pitch;
    g.comp = (long long)(nz + 1) * g.plane;

    int rc = FDTD_OK;
    auto fail = [&](int code) { release(h); return code; };
    for (int s = 0; s < 2; ++s) {
        if (cudaMalloc(&h->fields[s], field_bytes(h)) != cudaSuccess) { cudaGetLastError(); return fail(FDTD_ERR_OOM); }
        if ((rc = note(h, cudaMemsetAsync(h->fields[s], 0, field_bytes(h), h->stream))) != FDTD_OK) return fail(rc);
    }
    h->cur = 0;

    // CPML: coefficient tables and psi arrays over the slabs
    if (P > 0) {
        const int N[3] = {nx, ny, nz};
        size_t ncoef = 0;
        for (int a = 0; a < 3; ++a) ncoef += 4 * (size_t)(N[a] + 1);
        if (cudaMalloc(&h->coef_block, ncoef * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return fail(FDTD_ERR_OOM); }
        float *hc = (float *)std::calloc(ncoef, sizeof(float));
        if (!hc) return fail(FDTD_ERR_OOM);
        size_t off = 0;
        for (int a = 0; a < 3; ++a) {
            const size_t n1 = (size_t)N[a] + 1;
            float *aE = hc + off, *bE = aE + n1, *aH = bE + n1, *bH = aH + n1;
            cpml_coefficients(N[a], P, dx, dt, eps_r, aE, bE, aH, bH);
            h->aE[a] = h->coef_block + off;
            h->bE[a] = h->coef_block + off + n1;
            h->aH[a] = h->coef_block + off + 2 * n1;
            h->bH[a] = h->coef_block + off + 3 * n1;
            off += 4 * n1;
        }
        rc = note(h, cudaMemcpy(h->coef_block, hc, ncoef * sizeof(float), cudaMemcpyHostToDevice));
        std::free(hc);
        if (rc != FDTD_OK) return fail(rc);
        const int W = 2 * P + 1;
        const size_t pitch = (size_t)h->g.pitch;
        auto r32 = [](size_t n) { return (n + 31) / 32 * 32; };
        h->psi_axis[0] = r32((size_t)nz * ny * psi_x_row(nx, P));
        h->psi_axis[1] = r32((size_t)nz * W * pitch);
        h->psi_axis[2] = r32((size_t)W * ny * pitch);
        // E psi (2 per axis), then H psi set 0 and set 1 (2 per axis each)
        h->psi_floats = 3 * 2 * (h->psi_axis[0] + h->psi_axis[1] + h->psi_axis[2]);
        if (cudaMalloc(&h->psi_block, h->psi_floats * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return fail(FDTD_ERR_OOM); }
        if ((rc = note(h, cudaMemsetAsync(h->psi_block, 0, h->psi_floats * sizeof(float), h->stream))) != FDTD_OK) return fail(rc);
        const size_t third = h->psi_floats / 3 * sizeof(float);
        if (cudaMalloc(&h->epsi2, third) != cudaSuccess) { cudaGetLastError(); return fail(FDTD_ERR_OOM); }
        if ((rc = note(h, cudaMemsetAsync(h->epsi2, 0, third, h->stream))) != FDTD_OK) return fail(rc);
    }
    if (cudaMalloc(&h->d_flags, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return fail(FDTD_ERR_OOM); }
    if ((rc = note(h, cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream))) != FDTD_OK) return fail(rc);

    // scratch of the energy / stability reduction
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev);
    h->num_sms = sms > 0 ? sms : 1;
    h->partial_cap = sms > 0 ? 4 * sms : 512;
    if (cudaMalloc(&h->d_partial, 3 * (size_t)h->partial_cap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->d_result, 3 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(FDTD_ERR_OOM);
    }
    if ((rc = note(h, cudaStreamSynchronize(h->stream))) != FDTD_OK) return fail(rc);
    // default field-update path: two steps per pass where it applies (PEC and
    // CPML grids of at least FDTD_TWO_STEP_MIN_CELLS cells), else the one-step
    // vector-tile z-march; the others stay available (fdtd_set_kernel) as
    // cross-checks
    h->watch_every = FDTD_WATCHDOG_DEFAULT_STEPS;
    h->kernel = 0;
    if (vtile_prepare(h) == FDTD_OK) h->kernel = 1;
    if ((long long)nx * ny * nz >= FDTD_TWO_STEP_MIN_CELLS && tb2_prepare(h) == FDTD_OK) h->kernel = 2;
    cudaGetLastError();
    *out = h;
    return FDTD_OK;
}

void fdtd_destroy(fdtd_t h) { release(h); }

int fdtd_set_shower(fdtd_t h, const double *q, int n_bins, double z0, double bin_dz, int axis,
                    double v, const double *w, int L) {
    if (!h || !q || !w || n_bins < 2 || !(bin_dz > 0.0) || L < 0 || !std::isfinite(z0) ||
        !std::isfinite(v))
        return FDTD_ERR_ARG;
    if (axis != 2) return FDTD_ERR_ARG;
    const Grid &g = h->g;
    const int ic = g.nx / 2, jc = g.ny / 2, lo = interior_lo(h);
    if (ic - L < lo || ic + L > g.nx - lo || jc - L < lo || jc + L > g.ny - lo) return FDTD_ERR_ARG;
    for (int b = 0; b < n_bins; ++b) if (!std::isfinite(q[b])) return FDTD_ERR_ARG;
    const int nw = (2 * L + 1) * (2 * L + 1);
    for (int t = 0; t < nw; ++t) if (!std::isfinite(w[t])) return FDTD_ERR_ARG;
    TRY(h, cudaStreamSynchronize(h->stream));
    free_dev(h->d_q); h->d_q = nullptr;
    free_dev(h->d_w); h->d_w = nullptr;
    h->src.active = 0;
    if (cudaMalloc(&h->d_q, sizeof(double) * n_bins) != cudaSuccess ||
        cudaMalloc(&h->d_w, sizeof(double) * nw) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_OOM;
    }
    TRY(h, cudaMemcpy(h->d_q, q, sizeof(double) * n_bins, cudaMemcpyHostToDevice));
    TRY(h, cudaMemcpy(h->d_w, w, sizeof(double) * nw, cudaMemcpyHostToDevice));
    Source &s = h->src;
    s.L = L; s.ic = ic; s.jc = jc;
    s.kmin = h->boundary == FDTD_CPML ? h->P : 0;
    s.kmax = h->boundary == FDTD_CPML ? g.nz - h->P - 1 : g.nz - 1;
    s.nbins = n_bins;
    s.z0 = z0; s.v = v; s.dt = h->dt; s.dx = h->dx; s.bin_dz = bin_dz;
    s.coef = 1.0 / (h->eps * h->dx * h->dx);
    s.q = h->d_q; s.w = h->d_w;
    s.active = 1;
    return FDTD_OK;
}

int fdtd_clear_shower(fdtd_t h) {
    if (!h) return FDTD_ERR_ARG;
    h->src.active = 0;
    return FDTD_OK;
}

int fdtd_set_probes(fdtd_t h, const double *xyz, int n, int max_steps) {
    if (!h || n < 0 || max_steps < 0 || (n > 0 && !xyz)) return FDTD_ERR_ARG;
    const Grid &g = h->g;
    const int lo = interior_lo(h);
    std::vector<int> ijk(3 * (size_t)n);
    std::vector<float> cxy(2 * (size_t)n);
    for (int p = 0; p < n; ++p) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            double u = xyz[3 * p + a] / h->dx;
            if (!std::isfinite(u) || std::fabs(u) > 1e9) return FDTD_ERR_ARG;
            c[a] = (int)std::floor(u + 0.5);
        }
        if (c[0] < lo || c[0] > g.nx - lo || c[1] < lo || c[1] > g.ny - lo || c[2] < lo || c[2] > g.nz - lo)
            return FDTD_ERR_ARG;
        ijk[3 * p] = c[0]; ijk[3 * p + 1] = c[1]; ijk[3 * p + 2] = c[2];
        double X = (c[0] - g.nx / 2) * h->dx, Y = (c[1] - g.ny / 2) * h->dx;
        double r = std::sqrt(X * X + Y * Y);
        cxy[2 * p] = r > 0.0 ? (float)(X / r) : 0.0f;
        cxy[2 * p + 1] = r > 0.0 ? (float)(Y / r) : 0.0f;
    }
    TRY(h, cudaStreamSynchronize(h->stream));
    free_dev(h->d_ijk); free_dev(h->d_cxy); free_dev(h->d_trace);
    h->d_ijk = nullptr; h->d_cxy = nullptr; h->d_trace = nullptr;
    h->np = 0; h->max_steps = max_steps;
    h->probe_ver++;
    h->h_ijk.clear();
    if (n == 0) return FDTD_OK;
    size_t tb = sizeof(float) * 2 * (size_t)n * (size_t)(max_steps > 0 ? max_steps : 1);
    if (cudaMalloc(&h->d_ijk, sizeof(int) * 3 * n) != cudaSuccess ||
        cudaMalloc(&h->d_cxy, sizeof(float) * 2 * n) != cudaSuccess ||
        cudaMalloc(&h->d_trace, tb) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ERR_OOM;
    }
    TRY(h, cudaMemcpy(h->d_ijk, ijk.data(), sizeof(int) * 3 * n, cudaMemcpyHostToDevice));
    TRY(h, cudaMemcpy(h->d_cxy, cxy.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice));
    TRY(h, cudaMemset(h->d_trace, 0, tb));
    h->np = n;
    h->h_ijk = ijk;
    return FDTD_OK;
}

int fdtd_probe_nodes(fdtd_t h, int *ijk) {
    if (!h || (h->np > 0 && !ijk)) return FDTD_ERR_ARG;
    if (h->np) std::memcpy(ijk, h->h_ijk.data(), sizeof(int) * 3 * h->np);
    return FDTD_OK;
}

int fdtd_step(fdtd_t h, int n) {
    if (!h || n < 0) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    if (h->np > 0 && h->steps + n > h->max_steps) return FDTD_ERR_CAPACITY;
    return fdtd::fdtd_step_on(h, n, h->stream);
}

// Read the device error flags (after a synchronisation) into the sticky status.
static int check_flags(fdtd_ctx *h) {
    int f = 0;
    if (note(h, cudaMemcpy(&f, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost)) != FDTD_OK) return h->status;
    if (f != 0 && h->status == FDTD_OK)
        h->status = (f & ~fdtd::FLAG_UNSTABLE) ? FDTD_ERR_TIMEOUT : FDTD_ERR_UNSTABLE;
    return h->status;
}

int fdtd_sync(fdtd_t h) {
    if (!h) return FDTD_ERR_ARG;
    note(h, cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

int fdtd_steps_done(fdtd_t h, int64_t *steps) {
    if (!h || !steps) return FDTD_ERR_ARG;
    *steps = h->steps;
    return FDTD_OK;
}

int fdtd_probes(fdtd_t h, float *out, int on_device) {
    if (!h || (h->np > 0 && !out)) return FDTD_ERR_ARG;
    TRY(h, cudaStreamSynchronize(h->stream));
    if (check_flags(h) != FDTD_OK) return h->status;
    if (h->np == 0 || h->max_steps == 0) return FDTD_OK;
    size_t tb = sizeof(float) * 2 * (size_t)h->np * h->max_steps;
    TRY(h, cudaMemcpyAsync(out, h->d_trace, tb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           h->stream));
    TRY(h, cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

static size_t compact_bytes(const fdtd_ctx *h) {
    return sizeof(float) * (size_t)(h->g.nx + 1) * (h->g.ny + 1) * (h->g.nz + 1);
}

int fdtd_fields(fdtd_t h, int comp, float *out, int on_device) {
    if (!h || !out || comp < 0 || comp > 5) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    float *dst = out;
    if (!on_device) {
        if (cudaMalloc(&dst, compact_bytes(h)) != cudaSuccess) { cudaGetLastError(); return FDTD_ERR_OOM; }
    }
    launch_get_field(h, comp, dst, h->stream);
    h->launches++;
    int rc = note(h, cudaGetLastError());
    if (rc == FDTD_OK && !on_device)
        rc = note(h, cudaMemcpyAsync(out, dst, compact_bytes(h), cudaMemcpyDeviceToHost, h->stream));
    if (rc == FDTD_OK) rc = note(h, cudaStreamSynchronize(h->stream));
    if (!on_device) cudaFree(dst);
    return rc;
}

int fdtd_set_field(fdtd_t h, int comp, const float *in, int on_device) {
    if (!h || !in || comp < 0 || comp > 5) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    const float *src = in;
    float *tmp = nullptr;
    if (!on_device) {
        if (cudaMalloc(&tmp, compact_bytes(h)) != cudaSuccess) { cudaGetLastError(); return FDTD_ERR_OOM; }
        int rc = note(h, cudaMemcpyAsync(tmp, in, compact_bytes(h), cudaMemcpyHostToDevice, h->stream));
        if (rc != FDTD_OK) { cudaFree(tmp); return rc; }
        src = tmp;
    }
    launch_set_field(h, comp, src, h->stream);
    h->launches++;
    int rc = note(h, cudaGetLastError());
    if (rc == FDTD_OK) rc = note(h, cudaStreamSynchronize(h->stream));
    if (tmp) cudaFree(tmp);
    return rc;
}

int fdtd_reset(fdtd_t h) {
    if (!h) return FDTD_ERR_ARG;
    for (int s = 0; s < 2; ++s) TRY(h, cudaMemsetAsync(h->fields[s], 0, field_bytes(h), h->stream));
    if (h->psi_block) TRY(h, cudaMemsetAsync(h->psi_block, 0, h->psi_floats * sizeof(float), h->stream));
    if (h->epsi2) TRY(h, cudaMemsetAsync(h->epsi2, 0, h->psi_floats / 3 * sizeof(float), h->stream));
    h->ecur = 0;
    if (h->d_trace)
        TRY(h, cudaMemsetAsync(h->d_trace, 0, sizeof(float) * 2 * (size_t)h->np * h->max_steps, h->stream));
    h->cur = 0;
    h->steps = 0;
    if (h->status == FDTD_ERR_UNSTABLE) {
        // the non-finite values are gone with the fields: the handle is usable again
        TRY(h, cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream));
        h->status = FDTD_OK;
    }
    return note(h, cudaGetLastError());
}

int fdtd_energy(fdtd_t h, double *energy) {
    if (!h || !energy) return FDTD_ERR_ARG;
    if (h->status != FDTD_OK) return h->status;
    int nl = 0;
    launch_energy(h, h->stream, &nl);
    h->launches += nl;
    TRY(h, cudaGetLastError());
    double r[3];
    TRY(h, cudaMemcpyAsync(r, h->d_result, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    TRY(h, cudaStreamSynchronize(h->stream));
    const double v = h->dx * h->dx * h->dx;
    *energy = 0.5 * h->eps * r[0] * v + 0.5 * kMu0 * r[1] * v;
    return r[2] > 0.0 ? FDTD_ERR_UNSTABLE : FDTD_OK;
}

// ---- checkpoint --------------------------------------------------------------

namespace {
struct StateHeader {
    char magic[8];
    uint32_t version;
    int32_t nx, ny, nz, boundary, P, pitch, np, max_steps;
    int64_t steps;
    uint64_t field_bytes, psi_bytes, trace_bytes;
};
const char kMagic[8] = {'F', 'D', 'T', 'D', 'G', 'B', '3', 0};
}  // namespace

int fdtd_save_state(fdtd_t h, void *buf, size_t *bytes) {
    if (!h || !bytes) return FDTD_ERR_ARG;
    StateHeader hd{};
    std::memcpy(hd.magic, kMagic, 8);
    hd.version = 1;
    hd.nx = h->g.nx; hd.ny = h->g.ny; hd.nz = h->g.nz;
    hd.boundary = h->boundary; hd.P = h->P; hd.pitch = h->g.pitch;
    hd.np = h->np; hd.max_steps = h->max_steps; hd.steps = h->steps;
    hd.field_bytes = field_bytes(h);
    hd.psi_bytes = (h->psi_floats / 3) * 2 * sizeof(float);  // E psi + H psi of set cur
    hd.trace_bytes = h->np > 0 ? sizeof(float) * 2 * (size_t)h->np * h->max_steps : 0;
    size_t need = sizeof(hd) + hd.field_bytes + hd.psi_bytes + hd.trace_bytes;
    if (!buf) { *bytes = need; return FDTD_OK; }
    if (*bytes < need) return FDTD_ERR_ARG;
    TRY(h, cudaStreamSynchronize(h->stream));
    if (h->status != FDTD_OK) return h->status;
    char *p = (char *)buf;
    std::memcpy(p, &hd, sizeof(hd)); p += sizeof(hd);
    TRY(h, cudaMemcpy(p, h->fields[h->cur], hd.field_bytes, cudaMemcpyDeviceToHost)); p += hd.field_bytes;
    if (hd.psi_bytes) {
        const size_t third = h->psi_floats / 3 * sizeof(float);
        TRY(h, cudaMemcpy(p, h->ecur ? h->epsi2 : h->psi_block, third, cudaMemcpyDeviceToHost));
        TRY(h, cudaMemcpy(p + third, (char *)h->psi_block + third * (1 + h->cur), third, cudaMemcpyDeviceToHost));
        p += hd.psi_bytes;
    }
    if (hd.trace_bytes) { TRY(h, cudaMemcpy(p, h->d_trace, hd.trace_bytes, cudaMemcpyDeviceToHost)); }
    *bytes = need;
    return FDTD_OK;
}

int fdtd_load_state(fdtd_t h, const void *buf, size_t bytes) {
    if (!h || !buf || bytes < sizeof(StateHeader)) return FDTD_ERR_ARG;
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, kMagic, 8) != 0 || hd.version != 1) return FDTD_ERR_ARG;
    if (hd.nx != h->g.nx || hd.ny != h->g.ny || hd.nz != h->g.nz || hd.boundary != h->boundary ||
        hd.P != h->P || hd.pitch != h->g.pitch || hd.np != h->np || hd.max_steps != h->max_steps)
        return FDTD_ERR_ARG;
    if (hd.field_bytes != field_bytes(h) || hd.psi_bytes != (h->psi_floats / 3) * 2 * sizeof(float) ||
        bytes < sizeof(hd) + hd.field_bytes + hd.psi_bytes + hd.trace_bytes)
        return FDTD_ERR_ARG;
    TRY(h, cudaStreamSynchronize(h->stream));
    const char *p = (const char *)buf + sizeof(hd);
    TRY(h, cudaMemcpy(h->fields[h->cur], p, hd.field_bytes, cudaMemcpyHostToDevice)); p += hd.field_bytes;
    if (hd.psi_bytes) {
        const size_t third = h->psi_floats / 3 * sizeof(float);
        TRY(h, cudaMemcpy(h->psi_block, p, third, cudaMemcpyHostToDevice));
        h->ecur = 0;
        TRY(h, cudaMemcpy((char *)h->psi_block + third * (1 + h->cur), p + third, third, cudaMemcpyHostToDevice));
        p += hd.psi_bytes;
    }
    if (hd.trace_bytes) { TRY(h, cudaMemcpy(h->d_trace, p, hd.trace_bytes, cudaMemcpyHostToDevice)); }
    h->steps = hd.steps;
    return FDTD_OK;
}

// ---- instrumentation ----------------------------------------------------------

int fdtd_timing_begin(fdtd_t h, int max_launches) {
    if (!h || max_launches < 0) return FDTD_ERR_ARG;
    TimingRec &t = h->timing;
    while ((int)t.ev.size() < 2 * max_launches) {
        cudaEvent_t e;
        TRY(h, cudaEventCreate(&e));
        t.ev.push_back(e);
    }
    t.cap = max_launches;
    t.used = 0;
    t.on = true;
    return FDTD_OK;
}

int fdtd_timing_end(fdtd_t h, double *total_ms, int *launches) {
    if (!h || !total_ms || !launches) return FDTD_ERR_ARG;
    TimingRec &t = h->timing;
    t.on = false;
    TRY(h, cudaStreamSynchronize(h->stream));
    double tot = 0.0;
    for (int u = 0; u < t.used; ++u) {
        float ms = 0.0f;
        TRY(h, cudaEventElapsedTime(&ms, t.ev[2 * u], t.ev[2 * u + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *launches = t.used;
    return FDTD_OK;
}

int fdtd_timed_cells(fdtd_t h, int64_t *cells) {
    if (!h || !cells) return FDTD_ERR_ARG;
    const Grid &g = h->g;
    *cells = (int64_t)g.nx * g.ny * g.nz * (h->kernel == 2 ? 2 : 1);
    return FDTD_OK;
}

int fdtd_launch_count(fdtd_t h, int64_t *launches) {
    if (!h || !launches) return FDTD_ERR_ARG;
    *launches = h->launches;
    return FDTD_OK;
}

const char *fdtd_kernel_name(fdtd_t h) {
    if (h && h->kernel == 1) return vtile_name();
    if (h && h->kernel == 2) return tb2_name(h);
    return "unfused-h-then-e";
}

int fdtd_set_watchdog(fdtd_t h, int every) {
    if (!h || every < 0) return FDTD_ERR_ARG;
    h->watch_every = every;
    return FDTD_OK;
}

int fdtd_set_kernel(fdtd_t h, int which) {
    if (!h || which < 0 || which > 2) return FDTD_ERR_ARG;
    if (which == 1 && !h->vtile) return FDTD_ERR_ARG;
    if (which == 2 && !h->tb2) {
        if (h->boundary == FDTD_MUR1) return FDTD_ERR_ARG;
        const int rc = tb2_prepare(h);
        if (rc != FDTD_OK) return rc == FDTD_ERR_CUDA ? FDTD_ERR_CUDA : FDTD_ERR_ARG;
    }
    h->kernel = which;
    return FDTD_OK;
}

}  // extern "C"
