// The radial sweep of a polar disk, for dimensional splitting in two dimensions
// (Sec. 3.5): the plan's rows are the rings of one shared azimuthal mesh; every
// azimuthal column takes one flux-form upwind step in r in cylindrical geometry,
//   q'_j = q_j - dt (rf[j+1] F_{j+1} - rf[j] F_j) / A_j,  A_j = (rf[j+1]^2 - rf[j]^2)/2,
// with F = vr q_up (donor) or vr times the upwind ring's van Leer profile (the
// harmonic slope over the ring centres' spacings, Sec. 3.1; zero in the two rings
// next to the walls) at the midpoint of the swept interval, and closed walls
// (F = 0 on faces 0 and n_rows).  One thread per cell; neighbouring threads take
// neighbouring azimuthal cells of one ring, so every access is coalesced.  The
// geometry is formed in FP64 from the face radii.
#include <cuda_runtime.h>

#include "ram_device.cuh"

namespace ram {
namespace {

template <typename T>
__device__ __forceinline__ T ring_slope(const T *q, const double *rf, int nr, int N, int i, int k)
{
    if (k <= 0 || k >= nr - 1) return T(0);
    const T qm = q[(size_t)(k - 1) * N + i], q0 = q[(size_t)k * N + i], qp = q[(size_t)(k + 1) * N + i];
    const T hl = (T)(0.5 * (rf[k + 1] - rf[k - 1])), hr = (T)(0.5 * (rf[k + 2] - rf[k]));
    const T dl = Num<T>::div(q0 - qm, hl), dr = Num<T>::div(qp - q0, hr);
    const T pr = dl * dr;
    return pr > T(0) ? Num<T>::div(T(2) * pr, dl + dr) : T(0);
}

// flux through face f (radius rf[f], between rings f-1 and f) at azimuthal cell i
template <typename T>
__device__ __forceinline__ T face_flux(const T *q, const T *vr, const double *rf, int nr, int N,
                                       int i, int f, T dt, bool vl, bool &cfl_bad)
{
    if (f <= 0 || f >= nr) return T(0);
    const T v = vr[(size_t)f * N + i];
    const T c = v * dt;
    T qh = T(0);
    if (c > T(0)) {
        const int u = f - 1;
        const T w = (T)(rf[u + 1] - rf[u]);
        qh = q[(size_t)u * N + i];
        if (vl) qh += T(0.5) * ring_slope(q, rf, nr, N, i, u) * (w - c);
        cfl_bad |= c > w;
    } else if (c < T(0)) {
        const int u = f;
        const T w = (T)(rf[u + 1] - rf[u]);
        qh = q[(size_t)u * N + i];
        if (vl) qh -= T(0.5) * ring_slope(q, rf, nr, N, i, u) * (w + c);
        cfl_bad |= -c > w;
    }
    return v * qh;
}

template <typename T>
__global__ void __launch_bounds__(256) k_radial(int nr, int N, const T *q, T *out,
                                                const double *rf, const T *vr, double dt,
                                                int vl, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= N) return;
    bool bad = false;
    const T dtt = (T)dt;
    const T Fl = face_flux(q, vr, rf, nr, N, i, j, dtt, vl != 0, bad);
    const T Fu = face_flux(q, vr, rf, nr, N, i, j + 1, dtt, vl != 0, bad);
    const double area = 0.5 * (rf[j + 1] * rf[j + 1] - rf[j] * rf[j]);
    const T ka = (T)(dt / area);
    out[(size_t)j * N + i] = q[(size_t)j * N + i] - ka * ((T)rf[j + 1] * Fu - (T)rf[j] * Fl);
    if (bad) atomicOr(err, ERR_CFL);
}

}  // namespace

cudaError_t launch_radial(const Plan &p, ram_dtype dt, const void *q_in, void *q_out,
                          const double *rf, const void *vr, double step, int scheme,
                          cudaStream_t s)
{
    const int nr = p.n_rows;
    const int N = p.rows_h[0].n;
    const dim3 grid((N + 255) / 256, nr);
    if (dt == RAM_F32)
        k_radial<float><<<grid, 256, 0, s>>>(nr, N, static_cast<const float *>(q_in),
                                             static_cast<float *>(q_out), rf,
                                             static_cast<const float *>(vr), step,
                                             scheme == RAM_VANLEER, p.err);
    else
        k_radial<double><<<grid, 256, 0, s>>>(nr, N, static_cast<const double *>(q_in),
                                              static_cast<double *>(q_out), rf,
                                              static_cast<const double *>(vr), step,
                                              scheme == RAM_VANLEER, p.err);
    return cudaGetLastError();
}

}  // namespace ram
