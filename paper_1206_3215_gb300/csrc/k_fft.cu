// Plain batched row and column transforms: the 2D FFT that every time step
// is built from (Section 4), also exposed as pss_fft2d.
#include "launch.cuh"

namespace pss {

template <class Rl>
cudaError_t fft_rows(V2<Rl> *data, int64_t nx, int64_t rows_total, int dir, Rl scale,
                     const TW<Rl> *twx, cudaStream_t s)
{
    if (dir < 0) return launch_row<Rl>(nx, RowFft<Rl, -1>{data, scale}, twx, rows_total, s);
    return launch_row<Rl>(nx, RowFft<Rl, +1>{data, scale}, twx, rows_total, s);
}

template <class Rl>
cudaError_t fft_cols(V2<Rl> *data, int64_t nx, int64_t ny, int64_t batch, int dir, Rl scale,
                     const TW<Rl> *twy, cudaStream_t s)
{
    if (dir < 0) return launch_col<Rl>(ny, nx, ColFft<Rl, -1>{data, nx, scale}, twy, batch, s);
    return launch_col<Rl>(ny, nx, ColFft<Rl, +1>{data, nx, scale}, twy, batch, s);
}

template cudaError_t fft_rows<float>(float2 *, int64_t, int64_t, int, float, const float4 *,
                                     cudaStream_t);
template cudaError_t fft_rows<double>(double2 *, int64_t, int64_t, int, double, const double2 *,
                                      cudaStream_t);
template cudaError_t fft_cols<float>(float2 *, int64_t, int64_t, int64_t, int, float,
                                     const float4 *, cudaStream_t);
template cudaError_t fft_cols<double>(double2 *, int64_t, int64_t, int64_t, int, double,
                                      const double2 *, cudaStream_t);

}  // namespace pss
