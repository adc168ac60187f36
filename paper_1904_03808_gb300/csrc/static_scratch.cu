// static_scratch.cu -- allocation-free variant of the finest-level residual
// and restriction pair (mg_residual_restrict_static in include/qsmg.h).
//
// The fine-level residual that the allocating path keeps in a buffer made by
// mg_setup lives here in one fixed array compiled into the library.  Host
// code cannot use the array's name as a device address, so every call looks
// the address up with cudaGetSymbolAddress on the current device.  The lookup
// is not cached: after a cudaDeviceReset the module is loaded again, possibly
// at another address, and a cached pointer would be stale.
#include "../../include/qsmg.h"
#include "qsmg_impl.h"

using namespace qsmg;

namespace {

// 16 MiB: fine grids with 3 (nz+1) ny nx <= 2097152 corner values
constexpr long kStaticResidualDoubles = 2097152;

// every GPU that loads the library holds this array until the process exits
static __device__ __align__(256) double g_static_residual[kStaticResidualDoubles];

}  // namespace

extern "C" mg_status mg_residual_restrict_static(const mg_grid *grid, const mg_moduli *moduli,
                                                 const double *b, const double *x, double *bc,
                                                 void *stream) {
    if (!grid || !moduli || !b || !x || !bc) {
        set_last_error("mg_residual_restrict_static: null argument");
        return MG_ERR_ARG;
    }
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    if (nx < 4 || ny < 4 || nz < 2 || nx % 2 || ny % 2 || nz % 2) {
        set_last_error("mg_residual_restrict_static: grid %dx%dx%d unsupported "
                       "(nx, ny even >= 4; nz even >= 2)", nx, ny, nz);
        return MG_ERR_SHAPE;
    }
    const long need = 3L * (nz + 1) * ny * nx;
    if (need > kStaticResidualDoubles) {
        set_last_error("mg_residual_restrict_static: grid %dx%dx%d needs %ld residual values, the "
                       "static scratch holds %ld (16 MiB)", nx, ny, nz, need, kStaticResidualDoubles);
        return MG_ERR_SHAPE;
    }
    const double mu = moduli->mu, lam = moduli->K - 2.0 * mu / 3.0;
    if (!(mu > 0.0) || !(lam + mu > 0.0)) {
        set_last_error("mg_residual_restrict_static: need mu > 0 and lambda + mu > 0");
        return MG_ERR_ARG;
    }
    // the device address of the array in the current device's context
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_residual);
    if (e != cudaSuccess || !p) {
        set_last_error("mg_residual_restrict_static: cudaGetSymbolAddress: %s",
                       cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    double *r = (double *)p;
    // finest-level operator coefficients (scaled Eq. 30, stencils of section 3.4)
    Fine<double> f;
    f.lp = (lam + 2.0 * mu) / mu;
    f.kq = (lam + mu) / (4.0 * mu);
    f.d0 = 2.0 * f.lp + 4.0;
    f.dinv = 1.0 / f.d0;
    const Dims d = make_dims(nx, ny, nz);
    const Dims dc = make_dims(nx / 2, ny / 2, nz / 2);
    cudaStream_t st = (cudaStream_t)stream;
    // the residual kernel writes every interior value of r and zeroes its wall
    // planes, so nothing of the previous call's contents is read
    e = residual_fine(d, f, b, x, r, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bc, 0, 3 * (size_t)dc.cs * sizeof(double), st);
    if (e == cudaSuccess) e = restrict_fw(d, r, bc, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_last_error("mg_residual_restrict_static: %s", cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}
