// sisdc_solve_noalloc: the implicit solve without any allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code that runs under a fixed memory budget handed out by another
// framework's caching allocator, or a time-critical loop in which
// cudaMalloc's implicit device-wide synchronisation is not acceptable.  For
// them this entry point runs the same persistent PCG kernel as sisdc_solve,
// with all of its scratch (CG vectors, face traces, block partial sums,
// barrier words, tables) in one file-scope device array of fixed size that
// every GPU loading the library holds until the process exits.  The caller
// passes only the right-hand side and the solution.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>

#include "../../include/sisdc.h"
#include "ops.h"
#include "tables.h"

using namespace sisdc;

namespace {

// Fixed scratch: 16 MiB per device.
constexpr size_t kScratchDoubles = (size_t)SISDC_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
// device address of the array, per device; several host threads may look it
// up at once (they store the same value)
std::atomic<double*> s_scratch[kMaxDevices];

// Header layout (in doubles) at the start of the scratch array.
constexpr size_t H_BAR = 0;       // 2 unsigned (barrier arrival counter, exit counter)
constexpr size_t H_ERR = 1;       // int error flag
constexpr size_t H_ITERS = 2;     // int iteration count
constexpr size_t H_STATS = 4;     // ST_N long long
constexpr size_t H_SIZE = 32;     // header doubles (256 bytes)

int set_msg(char* buf, int len, const char* msg) {
    if (buf && len > 0) {
        std::strncpy(buf, msg, (size_t)len - 1);
        buf[len - 1] = '\0';
    }
    return 0;
}

}  // namespace

extern "C" sisdc_status sisdc_solve_noalloc(const sisdc_level_desc* d, int ncomp, double c, const double* d_rhs,
                                            double* d_x, double rtol, int maxit, void* cuda_stream, int* h_iters,
                                            char* h_err, int h_err_len) {
    set_msg(h_err, h_err_len, "");
    if (!d || !d_rhs || !d_x || !(c >= 0.0) || !(rtol > 0.0) || maxit < 1 ||
        (ncomp != 1 && ncomp != 2 && ncomp != 4)) {
        set_msg(h_err, h_err_len, "invalid argument");
        return SISDC_E_ARG;
    }
    if ((d->dim != 1 && d->dim != 2) || d->P < 1 || d->P > 8 || d->nel[0] < 1 ||
        (d->dim == 2 && d->nel[1] < 1) || !(d->hi[0] > d->lo[0]) || (d->dim == 2 && !(d->hi[1] > d->lo[1]))) {
        set_msg(h_err, h_err_len, "invalid level description");
        return SISDC_E_ARG;
    }
    const int nq = d->P + 1;
    const int ney = d->dim == 2 ? d->nel[1] : 1;
    const long long nel = (long long)d->nel[0] * ney;
    const int Q = d->dim == 2 ? nq * nq : nq;
    const long long NV = (long long)ncomp * nel * Q;
    const long long ntr = (long long)ncomp * nel * 2 * d->dim * 2 * nq;
    const size_t ntab = 2 * nq * nq + 3 * nq;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_msg(h_err, h_err_len, "no usable current CUDA device");
        return SISDC_E_CUDA;
    }
    // once per device, with that device current: the array's device address
    // (under lazy module loading this first lookup also loads the module and
    // commits the array on the device)
    double* base = s_scratch[dev].load(std::memory_order_acquire);
    if (!base) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_msg(h_err, h_err_len, "cudaGetSymbolAddress of the scratch array failed");
            return SISDC_E_CUDA;
        }
        base = static_cast<double*>(p);
        s_scratch[dev].store(base, std::memory_order_release);
    }

    // geometry and launch shape (no device memory needed for the query)
    const double hx = (d->hi[0] - d->lo[0]) / d->nel[0];
    const double hy = d->dim == 2 ? (d->hi[1] - d->lo[1]) / ney : 1.0;
    Geo g{};
    g.dim = d->dim; g.nq = nq; g.nqy = d->dim == 2 ? nq : 1; g.q = Q;
    g.nex = d->nel[0]; g.ney = ney; g.nel = (int)nel; g.ncomp = ncomp; g.N = nel * Q;
    g.hx = hx; g.hy = hy; g.taux = 2.0 * nq * nq / hx; g.tauy = 2.0 * nq * nq / hy;
    g.sx = 2.0 / hx; g.sy = 2.0 / hy; g.ihx = 1.0 / hx; g.ihy = 1.0 / hy;
    int block = 0;
    const int grid = pcg_grid(g, &block);
    if (grid < 1) {
        set_msg(h_err, h_err_len, "cooperative launch configuration unavailable");
        return SISDC_E_CUDA;
    }
    const size_t need = H_SIZE + ntab + 4 * (size_t)grid + 3 * (size_t)NV + 2 * (size_t)ntr;
    if (nel > (1LL << 30) || need > kScratchDoubles) {
        set_msg(h_err, h_err_len,
                "problem too large for the fixed scratch array (16 MiB: 5 NV doubles plus traces and tables)");
        return SISDC_E_ARG;
    }

    // host tables on the stack, copied into the scratch array
    double x[9], w[9], D[81], K[81], tab[2 * 81 + 27];
    if (!gll_tables_fixed(d->P, x, w, D, K)) {
        set_msg(h_err, h_err_len, "table construction failed");
        return SISDC_E_ARG;
    }
    for (int k = 0; k < nq * nq; ++k) { tab[k] = D[k]; tab[nq * nq + k] = K[k]; }
    for (int i = 0; i < nq; ++i) {
        tab[2 * nq * nq + i] = w[i];
        double dx = (2.0 / hx) * K[i * nq + i], dy = (2.0 / hy) * K[i * nq + i];
        if (i == nq - 1) { dx += -2.0 * D[nq * nq - 1] / hx + g.taux; dy += -2.0 * D[nq * nq - 1] / hy + g.tauy; }
        if (i == 0) { dx += 2.0 * D[0] / hx + g.taux; dy += 2.0 * D[0] / hy + g.tauy; }
        tab[2 * nq * nq + nq + i] = dx;
        tab[2 * nq * nq + 2 * nq + i] = dy;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* dtab = base + H_SIZE;
    double* part = dtab + ntab;
    double* r = part + 4 * (size_t)grid;
    double* p = r + NV;
    double* Ap = p + NV;
    double* trx = Ap + NV;
    double* trp = trx + ntr;
    // the array keeps the previous call's contents: clear what must start at zero
    e = cudaMemsetAsync(base, 0, H_SIZE * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dtab, tab, ntab * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_msg(h_err, h_err_len, cudaGetErrorString(e));
        return SISDC_E_CUDA;
    }
    g.D = dtab; g.K = dtab + nq * nq; g.w = dtab + 2 * nq * nq;
    g.dline_x = g.w + nq; g.dline_y = g.w + 2 * nq;

    PCGArgs a{};
    a.g = g;
    a.x = d_x;
    a.r = r; a.p = p; a.Ap = Ap; a.trx = trx; a.trp = trp;
    a.nterms = 1;
    a.in[0] = d_rhs;
    a.coef[0] = Coef{1.0, 0.0, nullptr};
    a.cimp = Coef{c, 0.0, nullptr};
    a.part = part;
    a.bar_count = reinterpret_cast<unsigned*>(base + H_BAR);
    a.bar_exit = a.bar_count + 1;
    a.err = reinterpret_cast<int*>(base + H_ERR);
    a.stats = reinterpret_cast<long long*>(base + H_STATS);
    a.rtol = rtol;
    a.maxit = maxit;
    a.iters_out = reinterpret_cast<int*>(base + H_ITERS);
    e = launch_pcg(a, grid, block, s);
    int flag = 0, iters = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, a.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&iters, a.iters_out, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_msg(h_err, h_err_len, cudaGetErrorString(e));
        return SISDC_E_CUDA;
    }
    if (h_iters) *h_iters = iters;
    if (flag & DEV_TIMEOUT) {
        set_msg(h_err, h_err_len, "a grid barrier wait timed out");
        return SISDC_E_TIMEOUT;
    }
    if (flag & DEV_NONFINITE) {
        set_msg(h_err, h_err_len, "non-finite value in the solve");
        return SISDC_E_NONFINITE;
    }
    if (flag & DEV_NOCONV) {
        set_msg(h_err, h_err_len, "the solve reached maxit");
        return SISDC_E_NOCONV;
    }
    return SISDC_OK;
}
