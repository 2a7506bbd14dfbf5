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
//   - Every call synchronises with its stream before it returns: it reads the step's
//     status back into host memory.
//   - The face coordinates come from the caller's device memory, so they are checked on
//     the device (see k_geo1d); a grid gq_fld_setup would reject returns
//     GQ_ERR_INVALID_ARG here too, with the fields untouched.
#include <cstring>
#include <mutex>

#include "gq_device.cuh"
#include "gq_geometry.cuh"
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

// The geometry formulas are gq_geometry.cuh's, which the plan's host set-up uses too.
// Caller-supplied faces are validated here as gq_fld_setup validates them on the host:
// finite and strictly increasing, r > 0 and theta within [0, pi] for spherical-polar
// grids, every volume positive and finite.  A violation sets bit 0 of the control
// block's input flags, so the solve does not run, the fields are left as they were and
// the call returns GQ_ERR_INVALID_ARG.

// 1-D geometry: dxf, thx, ymet (x-direction), dyf, thy (y-direction), and the face checks
__global__ void k_geo1d(int nx, int ny, int sph, const double* xf, const double* yf, DeviceGeometry g,
                        int* input_flags) {
    double* dxf = const_cast<double*>(g.dxf);
    double* thx = const_cast<double*>(g.thx);
    double* ymet = const_cast<double*>(g.ymet);
    double* dyf = const_cast<double*>(g.dyf);
    double* thy = const_cast<double*>(g.thy);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (t <= nx) {
        const int i = t;
        bad |= !isfinite(xf[i]) || (i > 0 && !(xf[i] > xf[i - 1])) || (sph && i == 0 && !(xf[0] > 0.0));
        if (i == 0) {
            dxf[0] = geom::x_centre(xf[0], xf[1], sph) - xf[0];
            thx[0] = 0.0;
        } else if (i == nx) {
            dxf[nx] = xf[nx] - geom::x_centre(xf[nx - 1], xf[nx], sph);
            thx[nx] = 0.0;
        } else {
            const double a = geom::x_centre(xf[i - 1], xf[i], sph), b = geom::x_centre(xf[i], xf[i + 1], sph);
            dxf[i] = b - a;
            thx[i] = (xf[i] - a) / (b - a);
        }
        if (i < nx) ymet[i] = sph ? geom::x_centre(xf[i], xf[i + 1], sph) : 1.0;
    }
    if (t <= ny) {
        const int j = t;
        bad |= !isfinite(yf[j]) || (j > 0 && !(yf[j] > yf[j - 1]));
        if (sph) bad |= (j == 0 && yf[0] < 0.0) || (j == ny && yf[ny] > geom::kPi + 1e-12);
        double dc;
        if (j == 0) {
            dyf[0] = geom::y_centre(yf[0], yf[1], sph, &dc) - yf[0];
            thy[0] = 0.0;
        } else if (j == ny) {
            dyf[ny] = yf[ny] - geom::y_centre(yf[ny - 1], yf[ny], sph, &dc);
            thy[ny] = 0.0;
        } else {
            const double a = geom::y_centre(yf[j - 1], yf[j], sph, &dc), b = geom::y_centre(yf[j], yf[j + 1], sph, &dc);
            dyf[j] = b - a;
            thy[j] = (yf[j] - a) / (b - a);
        }
    }
    if (bad) atomicOr(input_flags, 1);
}

// 2-D geometry: V per cell (checked positive and finite), A/d per x-face and y-face (uses
// the 1-D arrays)
__global__ void k_geo2d(int nx, int ny, int sph, const double* xf, const double* yf, DeviceGeometry g,
                        int* input_flags) {
    double* V = const_cast<double*>(g.V);
    double* gx = const_cast<double*>(g.gx);
    double* gy = const_cast<double*>(g.gy);
    const long long nxf = (long long)ny * (nx + 1), nyf = (long long)(ny + 1) * nx, N = (long long)nx * ny;
    bool bad = false;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N + nxf + nyf;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < N) {
            const int j = (int)(t / nx), i = (int)(t - (long long)j * nx);
            double dc;
            geom::y_centre(yf[j], yf[j + 1], sph, &dc);
            const double v = geom::cell_volume(xf[i], xf[i + 1], yf[j], yf[j + 1], sph, dc);
            bad |= !(v > 0.0) || !isfinite(v);
            V[t] = v;
        } else if (t < N + nxf) {
            const long long f = t - N;
            const int j = (int)(f / (nx + 1)), i = (int)(f - (long long)j * (nx + 1));
            double dc;
            geom::y_centre(yf[j], yf[j + 1], sph, &dc);
            gx[f] = geom::x_face_area(xf[i], yf[j], yf[j + 1], sph, dc) / g.dxf[i];
        } else {
            const long long f = t - N - nxf;
            const int j = (int)(f / nx), i = (int)(f - (long long)j * nx);
            gy[f] = geom::y_face_area(yf[j], xf[i], xf[i + 1], sph) / (g.ymet[i] * g.dyf[j]);
        }
    }
    if (bad) atomicOr(input_flags, 1);
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
    // the control block (whose input flags the geometry checks set) and the barrier word
    // must start at zero
    cudaError_t e = cudaMemsetAsync(P.ws.ctl, 0, sizeof(gq::SolveCtl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.ws.bar, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        gq::k_geo1d<<<(n1 + 255) / 256, 256, 0, st>>>(nx, ny, sph, x_faces, y_faces, P.geo, &P.ws.ctl->input_flags);
        gq::k_geo2d<<<std::max(1, std::min(sms * 8, (int)((3ll * P.N + 255) / 256))), 256, 0, st>>>(
            nx, ny, sph, x_faces, y_faces, P.geo, &P.ws.ctl->input_flags);
        e = cudaGetLastError();
    }
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
