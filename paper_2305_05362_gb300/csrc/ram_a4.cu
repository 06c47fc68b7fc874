// The fourth-order cell-average correction of Sec. 3.1 on uniform rows.
//
// The stored values are point values Q_i.  Before the remap they become the
// cell averages <Q>_i = Q_i + (Q_{i+1} - 2 Q_i + Q_{i-1}) / 24 (periodic), which the
// PPM remap moves; after it the point values are recovered from the remapped
// averages by inverting the same relation, Q_{i-1} + 22 Q_i + Q_{i+1} = 24 <Q>_i.
// That circulant system has the periodic Green's function
//   g_m = A (r^m + r^(N-m)) / (1 - r^N),  m = 0 .. N-1,
// with r = -11 + sqrt(120) (the root of r^2 + 22 r + 1 = 0 inside the unit circle)
// and A = 1 / (22 + 2 r), so Q_i = 24 sum_m g_m <Q>_{i+m}.  |r|^13 < 4e-18: for
// rows of 25 cells or more the sum is taken over |m| <= 12 on the infinite-lattice
// weights A r^|m| (the images are below FP64 rounding); shorter rows take the
// exact periodic weights.  Both kernels run one thread per cell over the plan's
// tiles of the order-3 uniform rows.
#include <cuda_runtime.h>

#include "ram_device.cuh"

namespace ram {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_a4_avg(const RowInfo *rows, const Tile *tiles,
                                                const T *q, T *avg)
{
    const Tile t = tiles[blockIdx.x];
    const RowInfo row = rows[t.row];
    const int N = row.n;
    const T *qr = q + row.cell_off;
    T *ar = avg + row.cell_off;
    for (int k = threadIdx.x; k < t.count; k += blockDim.x) {
        const int i = t.start + k;
        const T qm = qr[i > 0 ? i - 1 : N - 1], qp = qr[i + 1 < N ? i + 1 : 0];
        ar[i] = qr[i] + (qp - T(2) * qr[i] + qm) * (T(1) / T(24));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_a4_point(const RowInfo *rows, const Tile *tiles,
                                                  const T *avg, T *q)
{
    const Tile t = tiles[blockIdx.x];
    const RowInfo row = rows[t.row];
    const int N = row.n;
    const T *ar = avg + row.cell_off;
    T *qr = q + row.cell_off;
    const double r = -11.0 + sqrt(120.0);
    const double A = 1.0 / (22.0 + 2.0 * r);
    for (int k = threadIdx.x; k < t.count; k += blockDim.x) {
        const int i = t.start + k;
        T acc = T(0);
        if (N >= 25) {
            double w = A;  // A r^|m|
            acc = (T)w * ar[i];
            for (int m = 1; m <= 12; ++m) {
                w *= r;
                const int ip = i + m < N ? i + m : i + m - N;
                const int im = i - m >= 0 ? i - m : i - m + N;
                acc += (T)w * (ar[ip] + ar[im]);
            }
        } else {
            double rm = 1.0, rN = 1.0;
            for (int m = 0; m < N; ++m) rN *= r;
            double rNm = rN;  // r^(N - m), from m = 0
            const double inv = 1.0 / (1.0 - rN);
            for (int m = 0; m < N; ++m) {
                const double w = A * (rm + rNm) * inv;
                const int ip = i + m < N ? i + m : i + m - N;
                acc += (T)w * ar[ip];
                rm *= r;
                rNm /= r;
            }
        }
        qr[i] = T(24) * acc;
    }
}

template <typename T>
cudaError_t launch_a4_t(const Plan &p, const void *in, void *out, cudaStream_t s, bool to_avg)
{
    const int n = (int)p.tiles_uniform_h[3].size();
    if (n == 0) return cudaSuccess;
    if (to_avg)
        k_a4_avg<T><<<n, 256, 0, s>>>(p.rows, p.tiles_uniform[3], static_cast<const T *>(in),
                                      static_cast<T *>(out));
    else
        k_a4_point<T><<<n, 256, 0, s>>>(p.rows, p.tiles_uniform[3], static_cast<const T *>(in),
                                        static_cast<T *>(out));
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_a4(const Plan &p, ram_dtype dt, const void *in, void *out, cudaStream_t s,
                      bool to_avg)
{
    return dt == RAM_F32 ? launch_a4_t<float>(p, in, out, s, to_avg)
                         : launch_a4_t<double>(p, in, out, s, to_avg);
}

}  // namespace ram
