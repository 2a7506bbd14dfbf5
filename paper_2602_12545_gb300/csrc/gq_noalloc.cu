// Allocation-free variant of the single implicit FLD step.
//
// Some callers cannot allocate device memory: hosts whose device memory is carved up
// once at start-up and may not grow afterwards, plug-ins that live inside another
// application's memory manager (a raw cudaMalloc would bypass its accounting), and
// latency-bound loops that cannot afford cudaMalloc / cudaFree, which may synchronise
// the device.  gq_fld_step_noalloc serves them: all of the step's device
// scratch (geometry, set-up arrays, Krylov vectors, reductions, control block) lives in
// one statically sized __device__ array of this file, so the call allocates nothing.
// The caller still owns and passes the inputs and outputs (device pointers).
//
// Limits and rules:
//   - The array holds kNoAllocBytes (32 MiB) per device that loads the library, for the
//     life of the process.  Grids whose footprint exceeds it (about 50 000 cells) are
//     rejected with GQ_ERR_INVALID_ARG before anything runs.
//   - Every call on a device shares the one array, which keeps the previous call's
//     contents; the call clears what must start at zero.  Calls that overlap on the GPU
//     (two streams, or two host threads) race on the array: serialise them.
//   - The first call on a device resolves the array's device address with
//     cudaGetSymbolAddress (host code cannot use the symbol itself as a device pointer:
//     it names a host-side shadow).  Make that first call before any stream capture.
#include <cstring>
#include <mutex>

#include "gq_device.cuh"
#include "gq_internal.h"

namespace gq {
namespace {

constexpr size_t kNoAllocBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (resolved once per device)
cudaError_t scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// theta moments as in the plan's host geometry, on the device
__device__ void theta_moments_dev(double v, double h, double* first, double* zeroth) {
    double A, B;
    if (h < 0.05) {
        const double h2 = h * h;
        A = h2 * (0.5 + h2 * (-1.0 / 8.0 + h2 * (1.0 / 144.0 + h2 * (-1.0 / 5760.0))));
        B = h2 * h * (1.0 / 3.0 + h2 * (-1.0 / 30.0 + h2 * (1.0 / 840.0 + h2 * (-1.0 / 45360.0))));
    } else {
        A = cos(h) + h * sin(h) - 1.0;
        B = sin(h) - h * cos(h);
    }
    const double sv = sin(v), cv = cos(v), half = sin(0.5 * h);
    *first = sv * A + cv * B;
    *zeroth = sv * sin(h) + cv * 2.0 * half * half;
}

__device__ double xcen(const double* xf, int i, bool sph) {
    const double a = xf[i], b = xf[i + 1];
    return sph ? 0.75 * (a + b) * (a * a + b * b) / (a * a + a * b + b * b) : 0.5 * (a + b);
}

__device__ double ycen(const double* yf, int j, bool sph, double* dcos) {
    if (!sph) {
        *dcos = 1.0;
        return 0.5 * (yf[j] + yf[j + 1]);
    }
    double m1, m0;
    theta_moments_dev(yf[j], yf[j + 1] - yf[j], &m1, &m0);
    *dcos = m0;
    return yf[j] + m1 / m0;
}

// 1-D geometry: dxf, thx, ymet (x-direction), dyf, thy (y-direction)
__global__ void k_geo1d(int nx, int ny, int sph, const double* xf, const double* yf, DeviceGeometry g) {
    double* dxf = const_cast<double*>(g.dxf);
    double* thx = const_cast<double*>(g.thx);
    double* ymet = const_cast<double*>(g.ymet);
    double* dyf = const_cast<double*>(g.dyf);
    double* thy = const_cast<double*>(g.thy);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= nx) {
        const int i = t;
        if (i == 0) { dxf[0] = xcen(xf, 0, sph) - xf[0]; thx[0] = 0.0; }
        else if (i == nx) { dxf[nx] = xf[nx] - xcen(xf, nx - 1, sph); thx[nx] = 0.0; }
        else {
            const double a = xcen(xf, i - 1, sph), b = xcen(xf, i, sph);
            dxf[i] = b - a;
            thx[i] = (xf[i] - a) / (b - a);
        }
        if (i < nx) ymet[i] = sph ? xcen(xf, i, sph) : 1.0;
    }
    if (t <= ny) {
        const int j = t;
        double dc;
        if (j == 0) { dyf[0] = ycen(yf, 0, sph, &dc) - yf[0]; thy[0] = 0.0; }
        else if (j == ny) { dyf[ny] = yf[ny] - ycen(yf, ny - 1, sph, &dc); thy[ny] = 0.0; }
        else {
            const double a = ycen(yf, j - 1, sph, &dc), b = ycen(yf, j, sph, &dc);
            dyf[j] = b - a;
            thy[j] = (yf[j] - a) / (b - a);
        }
    }
}

// 2-D geometry: V per cell, A/d per x-face and y-face (uses the 1-D arrays)
__global__ void k_geo2d(int nx, int ny, int sph, const double* xf, const double* yf, DeviceGeometry g) {
    double* V = const_cast<double*>(g.V);
    double* gx = const_cast<double*>(g.gx);
    double* gy = const_cast<double*>(g.gy);
    const long long nxf = (long long)ny * (nx + 1), nyf = (long long)(ny + 1) * nx, N = (long long)nx * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N + nxf + nyf;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < N) {
            const int j = (int)(t / nx), i = (int)(t - (long long)j * nx);
            const double a = xf[i], b = xf[i + 1];
            double dc = 1.0;
            if (sph) ycen(yf, j, true, &dc);
            V[t] = sph ? (b - a) * (a * a + a * b + b * b) / 3.0 * dc : (b - a) * (yf[j + 1] - yf[j]);
        } else if (t < N + nxf) {
            const long long f = t - N;
            const int j = (int)(f / (nx + 1)), i = (int)(f - (long long)j * (nx + 1));
            double dc = 1.0;
            if (sph) ycen(yf, j, true, &dc);
            const double A = sph ? xf[i] * xf[i] * dc : yf[j + 1] - yf[j];
            gx[f] = A / g.dxf[i];
        } else {
            const long long f = t - N - nxf;
            const int j = (int)(f / nx), i = (int)(f - (long long)j * nx);
            double sf = 1.0;
            if (sph) sf = (yf[j] <= 0.0 || yf[j] >= M_PI) ? 0.0 : sin(yf[j]);
            const double a = xf[i], b = xf[i + 1];
            const double A = sph ? sf * (b - a) * (b + a) * 0.5 : b - a;
            gy[f] = A / (g.ymet[i] * g.dyf[j]);
        }
    }
}

}  // namespace
}  // namespace gq

extern "C" {

size_t gq_fld_step_noalloc_max_bytes(void) { return gq::kNoAllocBytes; }

gq_status gq_fld_step_noalloc(int nx, int ny, int coord, const double* x_faces, const double* y_faces,
                              const double* rho, double* e_g, double* E_r, double* T_g_out,
                              const gq_opacity_law* opacity, const gq_eos* eos, double dt, const gq_bc* bc,
                              const gq_solver_opts* opts, void* stream, gq_step_info* info) {
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = GQ_ERR_INVALID_ARG;
    }
    if (nx < 1 || ny < 1 || (long long)nx * ny > gq::kMaxCells || !x_faces || !y_faces) return GQ_ERR_INVALID_ARG;
    if (coord != GQ_CARTESIAN && coord != GQ_SPHERICAL_POLAR) return GQ_ERR_INVALID_ARG;
    int dev = -1, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GQ_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GQ_ERR_CUDA;
    const int per_sm = gq::solve_max_blocks_per_sm();
    if (per_sm < 1) return GQ_ERR_CUDA;
    gq_fld_plan P{};
    P.nx = nx;
    P.ny = ny;
    P.N = nx * ny;
    P.coord = coord;
    P.device = dev;
    P.num_sms = sms;
    const int need = (P.N + gq::kSolveThreads - 1) / gq::kSolveThreads;
    P.solve_grid_max = std::max(1, std::min(per_sm * sms, need));
    P.setup_blocks = std::max(1, std::min(sms * 8, (P.N + gq::kSetupThreads - 1) / gq::kSetupThreads));
    // size check before anything is enqueued
    const size_t bytes = gq::plan_layout(&P, nullptr);
    if (bytes > gq::kNoAllocBytes) return GQ_ERR_INVALID_ARG;

    gq::StepParams sp{};
    gq::SolveParams pp{};
    gq_status vs = gq::make_step_params(&P, rho, e_g, E_r, T_g_out, opacity, eos, dt, bc, opts, &sp, &pp, nullptr);
    if (vs != GQ_OK) return vs;

    void* base = nullptr;
    if (gq::scratch_address(dev, &base) != cudaSuccess) {
        cudaGetLastError();
        return GQ_ERR_CUDA;
    }
    gq::plan_layout(&P, static_cast<char*>(base));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sph = coord == GQ_SPHERICAL_POLAR;
    const int n1 = std::max(nx, ny) + 1;
    gq::k_geo1d<<<(n1 + 255) / 256, 256, 0, st>>>(nx, ny, sph, x_faces, y_faces, P.geo);
    gq::k_geo2d<<<std::max(1, std::min(sms * 8, (int)((3ll * P.N + 255) / 256))), 256, 0, st>>>(
        nx, ny, sph, x_faces, y_faces, P.geo);
    cudaError_t e = cudaGetLastError();
    // the control block and the barrier word must start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(P.ws.ctl, 0, sizeof(gq::SolveCtl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.ws.bar, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = gq::launch_setup(sp, P.geo, P.ws, P.setup_blocks, st);
    if (e == cudaSuccess) e = gq::launch_solve(pp, P.ws, P.solve_grid_max, st);
    if (e == cudaSuccess) e = gq::launch_backsub(sp, P.geo, P.ws, P.setup_blocks, st);
    gq::SolveCtl c{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, P.ws.ctl, sizeof(c), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (info) info->status = GQ_ERR_CUDA;
        return GQ_ERR_CUDA;
    }
    const gq_status status = gq::status_of(c);
    if (info) {
        gq::fill_info(c, status, info);
        info->solve_blocks = P.solve_grid_max;
    }
    return status;
}

}  // extern "C"
