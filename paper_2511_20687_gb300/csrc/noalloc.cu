// osam_hex8_force_noalloc: the internal force with the deterministic element-buffer scatter, for
// callers that may not allocate device memory.  The element buffer lives in a fixed file-scope
// device array instead of memory obtained from cudaMalloc.
//
// Who needs this: a host application that freezes its GPU memory budget after start-up and forbids
// further cudaMalloc / cudaFree (those calls can synchronise the device and fragment a pool the
// application manages itself), code that runs inside another allocator's hooks, and code on a thread
// that must never block on the implicit synchronisation cudaFree performs.  Such callers still pass
// their own input and output arrays; the only working memory used here is the static array below.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "osam.h"
#include "osam_internal.h"

namespace {

// 24 element contributions per element, OSAM_NOALLOC_MAX_ELEMENTS elements: 6 MiB of FP64.  The CUDA
// runtime loads this file's module (and with it the array) lazily: on a device, the memory is taken
// by the set-up of the first call (below), then held until the process exits.
__device__ __align__(256) double g_noalloc_fe[24LL * OSAM_NOALLOC_MAX_ELEMENTS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_fe_addr[kMaxDevices] = {nullptr};

// nodal force, interleaved output f[3 n + c], gathered from the element buffer in a fixed order
__global__ void k_gather_aos(int nx, int ny, int nz, const double* __restrict__ fe, double* __restrict__ f) {
    const int nn = (nx + 1) * (ny + 1) * (nz + 1);
    const int ne = nx * ny * nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nn) return;
    const int n = t / 3, c = t % 3;
    const int i = n % (nx + 1);
    const int q = n / (nx + 1);
    const int j = q % (ny + 1), k = q / (ny + 1);
    double s = 0.0;
    for (int az = 0; az < 2; ++az) {
        const int ke = k - az;
        if (ke < 0 || ke >= nz) continue;
        for (int ay = 0; ay < 2; ++ay) {
            const int je = j - ay;
            if (je < 0 || je >= ny) continue;
            for (int ax = 0; ax < 2; ++ax) {
                const int ie = i - ax;
                if (ie < 0 || ie >= nx) continue;
                const int e = ie + nx * (je + ny * ke);
                s += fe[(long long)((ax + 2 * ay + 4 * az) * 3 + c) * ne + e];
            }
        }
    }
    f[t] = s;
}

// Set-up of a device, once, with that device current: look up the device address of the static
// element buffer and run every kernel this entry point can launch once (each material's force and the
// gather) on a one-element mesh carved out of the same buffer.  Under the runtime's lazy loading, the
// first use of a module or kernel loads its code and may take device memory (the module's __device__
// array, kernel code, a larger local-memory reservation) and synchronise; doing all of it here keeps
// later calls free of that.  The warm-up results are never read: every call overwrites the buffer.
int device_setup(cudaStream_t s, double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        osam::set_thread_error("osam_hex8_force_noalloc: no current CUDA device");
        return OSAM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_fe_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_fe);
        if (e != cudaSuccess || !p) {
            osam::set_thread_error(std::string("osam_hex8_force_noalloc: cudaGetSymbolAddress failed: ") +
                                   cudaGetErrorString(e));
            return OSAM_ECUDA;
        }
        double* base = static_cast<double*>(p);
        // one element: element buffer at [0, 24), its 8 nodes' u at [24, 48), f at [48, 72)
        osam::ElemArgs a{};
        a.nx = a.ny = a.nz = a.ne = 1;
        a.invh = 1.0; a.w8 = 0.125; a.wq = 1.0 / 32.0; a.wq3 = 1.0 / 96.0; a.lam = 1.0; a.mu = 1.0;
        a.u = base + 24; a.usn = 3; a.usc = 1;
        a.fe = base;
        for (int m : {OSAM_LINEAR_ELASTIC, OSAM_NEO_HOOKEAN, OSAM_SAINT_VENANT_KIRCHHOFF})
            if (e == cudaSuccess) e = osam::launch_hex8_force(m, false, osam::kGather, a, s);
        if (e == cudaSuccess) {
            k_gather_aos<<<1, 32, 0, s>>>(1, 1, 1, base, base + 48);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            osam::set_thread_error(std::string("osam_hex8_force_noalloc: device set-up failed: ") +
                                   cudaGetErrorString(e));
            return OSAM_ECUDA;
        }
        g_fe_addr[dev] = base;
    }
    *out = g_fe_addr[dev];
    return OSAM_OK;
}

}  // namespace

extern "C" OSAM_API int osam_hex8_force_noalloc(int nx, int ny, int nz, double h, int material, double lambda,
                                                double mu, const double* lambda_e, const double* mu_e, const double* u,
                                                double* f, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !u || !f ||
        (material != OSAM_LINEAR_ELASTIC && material != OSAM_NEO_HOOKEAN && material != OSAM_SAINT_VENANT_KIRCHHOFF)) {
        osam::set_thread_error("osam_hex8_force_noalloc: invalid argument");
        return OSAM_EINVAL;
    }
    // each dimension is bounded first, so the element count below cannot overflow
    if (nx > OSAM_NOALLOC_MAX_ELEMENTS || ny > OSAM_NOALLOC_MAX_ELEMENTS || nz > OSAM_NOALLOC_MAX_ELEMENTS) {
        osam::set_thread_error("osam_hex8_force_noalloc: a mesh dimension exceeds the static buffer limit of " +
                               std::to_string(OSAM_NOALLOC_MAX_ELEMENTS) + " elements");
        return OSAM_EINVAL;
    }
    const long long ne = (long long)nx * ny * nz;
    if (ne > OSAM_NOALLOC_MAX_ELEMENTS) {
        osam::set_thread_error("osam_hex8_force_noalloc: " + std::to_string(ne) +
                               " elements exceed the static buffer limit of " +
                               std::to_string(OSAM_NOALLOC_MAX_ELEMENTS));
        return OSAM_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* fe = nullptr;
    if (int rc = device_setup(s, &fe)) return rc;
    osam::ElemArgs a{};
    a.nx = nx; a.ny = ny; a.nz = nz; a.ne = (int)ne;
    a.invh = 1.0 / h;
    a.w8 = h * h / 8.0;
    a.wq = h * h / 32.0;
    a.wq3 = h * h / 96.0;
    a.lam = lambda; a.mu = mu;
    a.lam_e = lambda_e; a.mu_e = mu_e;
    a.u = u; a.usn = 3; a.usc = 1;
    a.fe = fe;
    // every element writes all 24 of its entries, so the buffer needs no clearing between calls
    cudaError_t e = osam::launch_hex8_force(material, false, osam::kGather, a, s);
    if (e == cudaSuccess) {
        const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
        k_gather_aos<<<(int)((3 * nn + 255) / 256), 256, 0, s>>>(nx, ny, nz, fe, f);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        osam::set_thread_error(std::string("osam_hex8_force_noalloc: ") + cudaGetErrorString(e));
        return OSAM_ECUDA;
    }
    return OSAM_OK;
}
