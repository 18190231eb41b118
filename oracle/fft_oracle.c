/*
 * FP64 CPU oracle for the staged 3D FFT -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * this library. It shares no code, header, table or helper with the CUDA
 * library: it is a plain, slow, obviously-correct restatement of the
 * transforms the paper defines.
 *
 * What it computes (paper, Section III-A):
 *   A^(kx,ky,kz) = sum_{i,j,l} A(i,j,l) exp(-2 pi i (kx i/Nx + ky j/Ny + kz l/Nz))
 * evaluated separably, as the paper's pencil sequence does: 1D transforms
 * along x for all (y,z), then along y, then along z (Section III-A list,
 * Algorithm 1). The 1D transform is either
 *   - the naive O(n^2) DFT straight from the definition, or
 *   - a recursive decimation-in-time mixed-radix Cooley-Tukey FFT that splits
 *     off a factor 2, 3 or 5 and falls back to the naive DFT for any other
 *     (prime) length.
 * Twiddles are exp(sign * 2 pi i * (t mod n) / n) from libm cos/sin in FP64,
 * with the integer argument reduced first.
 *
 * Arrays are row-major [batch][z][y][x] (x fastest) of interleaved complex128
 * (re, im) doubles, the same element order as the paper's column-major
 * A(i,j,l) with i = x fastest.
 *
 * Threads: the pencils of one axis are split across `nthreads` POSIX threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846264338327950288

typedef struct {
    double re, im;
} cplx;

/* ---------------------------------------------------------------- twiddles */

/* Table w[t] = exp(sign * 2 pi i t / n), t in [0, n). */
static cplx* make_table(long n, int sign) {
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
    if (!w) return NULL;
    for (long t = 0; t < n; ++t) {
        double a = 2.0 * OR_PI * (double)t / (double)n;
        w[t].re = cos(a);
        w[t].im = (double)sign * sin(a);
    }
    return w;
}

static inline cplx cmul(cplx a, cplx b) {
    cplx r;
    r.re = a.re * b.re - a.im * b.im;
    r.im = a.re * b.im + a.im * b.re;
    return r;
}

/* ----------------------------------------------------------- 1D transforms */

/*
 * Naive DFT of length n: y[k] = sum_j x[j*xs] W^(j k), W = exp(sign 2 pi i/N0)^d
 * where the table holds the N0-th roots and d = N0 / n.
 */
static void dft_naive(const cplx* x, long xs, cplx* y, long n, const cplx* w, long n0) {
    long d = n0 / n;
    for (long k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (long j = 0; j < n; ++j) {
            long t = ((j * k) % n) * d;
            cplx v = cmul(x[j * xs], w[t]);
            sr += v.re;
            si += v.im;
        }
        y[k].re = sr;
        y[k].im = si;
    }
}

static long small_factor(long n) {
    if (n % 2 == 0) return 2;
    if (n % 3 == 0) return 3;
    if (n % 5 == 0) return 5;
    return 0;
}

/*
 * Recursive DIT FFT: y[k] = sum_j x[j*xs] W_n^(j k), y contiguous.
 * Split n = p*m: Y_q[k] = sum_s x[(q + p s) xs] W_m^(s k) for q < p, then
 * X[k + m t] = sum_q W_n^(q (k + m t)) Y_q[k].
 */
static void fft_rec(const cplx* x, long xs, cplx* y, long n, const cplx* w, long n0) {
    if (n == 1) {
        y[0] = x[0];
        return;
    }
    long p = small_factor(n);
    if (p == 0) {
        dft_naive(x, xs, y, n, w, n0);
        return;
    }
    long m = n / p;
    for (long q = 0; q < p; ++q) fft_rec(x + q * xs, xs * p, y + q * m, m, w, n0);
    long d = n0 / n;
    cplx tmp[5];
    for (long k = 0; k < m; ++k) {
        for (long q = 0; q < p; ++q) tmp[q] = y[q * m + k];
        for (long t = 0; t < p; ++t) {
            double sr = 0.0, si = 0.0;
            for (long q = 0; q < p; ++q) {
                long e = ((q * (k + m * t)) % n) * d;
                cplx v = cmul(tmp[q], w[e]);
                sr += v.re;
                si += v.im;
            }
            y[k + m * t].re = sr;
            y[k + m * t].im = si;
        }
    }
}

/* ------------------------------------------------------ batched pencil driver */

typedef struct {
    cplx* data;      /* array being transformed in place */
    long len;        /* transform length */
    long stride;     /* element stride along the transform axis */
    long n_pencils;  /* pencils = product of the other axes (and batch) */
    /* pencil index q -> base offset: q = (o * ninner + i): base = o*so + i*si */
    long ninner, si, so;
    const cplx* w;
    int naive;
    long first, last; /* pencil range for this worker */
} axis_job;

static void* axis_worker(void* arg) {
    axis_job* j = (axis_job*)arg;
    cplx* in = (cplx*)malloc(sizeof(cplx) * (size_t)j->len);
    cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)j->len);
    if (!in || !out) {
        free(in);
        free(out);
        return (void*)1;
    }
    for (long q = j->first; q < j->last; ++q) {
        long o = q / j->ninner, i = q % j->ninner;
        cplx* base = j->data + o * j->so + i * j->si;
        for (long t = 0; t < j->len; ++t) in[t] = base[t * j->stride];
        if (j->naive)
            dft_naive(in, 1, out, j->len, j->w, j->len);
        else
            fft_rec(in, 1, out, j->len, j->w, j->len);
        for (long t = 0; t < j->len; ++t) base[t * j->stride] = out[t];
    }
    free(in);
    free(out);
    return NULL;
}

/* Transform every pencil along one axis, in place. Returns 0 on success. */
static int run_axis(cplx* data, long len, long stride, long ninner, long si, long nouter, long so,
                    int sign, int naive, int nthreads) {
    if (len <= 1) return 0;
    cplx* w = make_table(len, sign);
    if (!w) return -1;
    long npen = ninner * nouter;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (npen < nthreads) nthreads = (int)(npen > 0 ? npen : 1);
    pthread_t th[256];
    axis_job jobs[256];
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].data = data;
        jobs[t].len = len;
        jobs[t].stride = stride;
        jobs[t].n_pencils = npen;
        jobs[t].ninner = ninner;
        jobs[t].si = si;
        jobs[t].so = so;
        jobs[t].w = w;
        jobs[t].naive = naive;
        jobs[t].first = npen * t / nthreads;
        jobs[t].last = npen * (t + 1) / nthreads;
    }
    if (nthreads == 1) {
        if (axis_worker(&jobs[0])) rc = -1;
    } else {
        int started = 0;
        for (int t = 0; t < nthreads; ++t) {
            if (pthread_create(&th[t], NULL, axis_worker, &jobs[t]) != 0) {
                rc = -1;
                break;
            }
            ++started;
        }
        for (int t = 0; t < started; ++t) {
            void* r = NULL;
            pthread_join(th[t], &r);
            if (r) rc = -1;
        }
    }
    free(w);
    return rc;
}

/* ------------------------------------------------------------- public API */

/*
 * 1D transform of `count` contiguous rows of length n (in place).
 * sign = -1 forward, +1 unscaled inverse. naive != 0 selects the O(n^2) DFT.
 */
int oracle_fft1d(double* data, long n, long count, int sign, int naive, int nthreads) {
    return run_axis((cplx*)data, n, 1, count, n, 1, 0, sign, naive, nthreads);
}

/*
 * Separable 3D C2C transform (unscaled), in place, on [batch][nz][ny][nx]:
 * x pencils, then y pencils, then z pencils (the paper's stage order).
 * `order` = 0 for x,y,z; 1 for z,y,x (used only to check axis-order
 * independence).
 */
int oracle_fft3d(double* data, long nx, long ny, long nz, long batch, int sign, int naive, int order,
                 int nthreads) {
    cplx* d = (cplx*)data;
    long plane = nx * ny, vol = plane * nz;
    for (int s = 0; s < 3; ++s) {
        int axis = order == 0 ? s : 2 - s;
        int rc = 0;
        if (axis == 0) /* x: rows contiguous; pencils indexed by (b,z,y) */
            rc = run_axis(d, nx, 1, ny * nz * batch, nx, 1, 0, sign, naive, nthreads);
        else if (axis == 1) /* y: stride nx; pencils (b,z) outer, x inner */
            rc = run_axis(d, ny, nx, nx, 1, nz * batch, plane, sign, naive, nthreads);
        else /* z: stride nx*ny; pencils b outer, (y,x) inner */
            rc = run_axis(d, nz, plane, plane, 1, batch, vol, sign, naive, nthreads);
        if (rc) return rc;
    }
    return 0;
}

/*
 * R2C forward: out[b][z][y][kx] for kx in [0, nx/2] = the first nx/2+1 x-bins
 * of the full C2C transform of the real input promoted to complex.
 * `in` is real [batch][nz][ny][nx]; `out` complex [batch][nz][ny][nx/2+1].
 */
int oracle_rfft3d(const double* in, double* out, long nx, long ny, long nz, long batch, int nthreads) {
    long nxc = nx / 2 + 1;
    long rows = ny * nz * batch;
    cplx* full = (cplx*)malloc(sizeof(cplx) * (size_t)(nx * rows));
    if (!full) return -1;
    for (long r = 0; r < rows; ++r)
        for (long x = 0; x < nx; ++x) {
            full[r * nx + x].re = in[r * nx + x];
            full[r * nx + x].im = 0.0;
        }
    int rc = run_axis(full, nx, 1, rows, nx, 1, 0, -1, 0, nthreads);
    cplx* o = (cplx*)out;
    if (!rc)
        for (long r = 0; r < rows; ++r) memcpy(o + r * nxc, full + r * nx, sizeof(cplx) * (size_t)nxc);
    free(full);
    if (rc) return rc;
    long plane = nxc * ny;
    rc = run_axis(o, ny, nxc, nxc, 1, nz * batch, plane, -1, 0, nthreads);
    if (rc) return rc;
    return run_axis(o, nz, plane, plane, 1, batch, plane * nz, -1, 0, nthreads);
}

/*
 * Unscaled C2R: the real part of the unscaled inverse C2C transform of the
 * Hermitian-completed full spectrum. For kx in (0, nx/2) the completion is
 * X[-k] = conj(X[k]); on the kx = 0 and kx = nx/2 planes the given half
 * spectrum is first projected onto its Hermitian part,
 * h(ky,kz) <- (h(ky,kz) + conj(h(-ky,-kz))) / 2.
 * `in` complex [batch][nz][ny][nx/2+1]; `out` real [batch][nz][ny][nx].
 */
int oracle_irfft3d(const double* in, double* out, long nx, long ny, long nz, long batch, int nthreads) {
    long nxc = nx / 2 + 1, M = nx / 2;
    long vol = nx * ny * nz;
    const cplx* h = (const cplx*)in;
    cplx* full = (cplx*)malloc(sizeof(cplx) * (size_t)(vol * batch));
    if (!full) return -1;
    for (long b = 0; b < batch; ++b) {
        const cplx* hb = h + b * nxc * ny * nz;
        cplx* fb = full + b * vol;
        for (long z = 0; z < nz; ++z)
            for (long y = 0; y < ny; ++y) {
                long zm = (nz - z) % nz, ym = (ny - y) % ny;
                for (long kx = 0; kx < nx; ++kx) {
                    cplx v;
                    if (kx == 0 || (kx == M && nx % 2 == 0)) {
                        cplx a = hb[(z * ny + y) * nxc + kx];
                        cplx c = hb[(zm * ny + ym) * nxc + kx];
                        v.re = 0.5 * (a.re + c.re);
                        v.im = 0.5 * (a.im - c.im);
                    } else if (kx <= M) {
                        v = hb[(z * ny + y) * nxc + kx];
                    } else {
                        cplx c = hb[(zm * ny + ym) * nxc + (nx - kx)];
                        v.re = c.re;
                        v.im = -c.im;
                    }
                    fb[(z * ny + y) * nx + kx] = v;
                }
            }
    }
    int rc = oracle_fft3d((double*)full, nx, ny, nz, batch, +1, 0, 0, nthreads);
    if (!rc)
        for (long i = 0; i < vol * batch; ++i) out[i] = full[i].re;
    free(full);
    return rc;
}

/*
 * Direct triple-sum DFT at selected bins (the definition, no factorisation):
 * out[q] = sum_{x,y,z} in[z][y][x] exp(sign 2 pi i (kx x/nx + ky y/ny + kz z/nz))
 * for bins[q] = (kx, ky, kz). One grid (no batch).
 */
int oracle_dft3d_bins(const double* in, long nx, long ny, long nz, const long* bins, long nbins,
                      int sign, double* out) {
    const cplx* a = (const cplx*)in;
    cplx* wx = make_table(nx, sign);
    cplx* wy = make_table(ny, sign);
    cplx* wz = make_table(nz, sign);
    if (!wx || !wy || !wz) {
        free(wx);
        free(wy);
        free(wz);
        return -1;
    }
    for (long q = 0; q < nbins; ++q) {
        long kx = bins[3 * q], ky = bins[3 * q + 1], kz = bins[3 * q + 2];
        double sr = 0.0, si = 0.0;
        for (long z = 0; z < nz; ++z) {
            cplx ez = wz[(kz * z) % nz];
            for (long y = 0; y < ny; ++y) {
                cplx eyz = cmul(wy[(ky * y) % ny], ez);
                const cplx* row = a + (z * ny + y) * nx;
                for (long x = 0; x < nx; ++x) {
                    cplx v = cmul(row[x], cmul(wx[(kx * x) % nx], eyz));
                    sr += v.re;
                    si += v.im;
                }
            }
        }
        out[2 * q] = sr;
        out[2 * q + 1] = si;
    }
    free(wx);
    free(wy);
    free(wz);
    return 0;
}

/*
 * The same direct triple sum as oracle_dft3d_bins, for a complex64 grid (each
 * value upcast to FP64 exactly as it is read, so a 2^30-point grid needs no
 * FP64 copy) with the bins split across `nthreads` POSIX threads. Per bin the
 * terms are added in the same order, so the results equal oracle_dft3d_bins
 * on the upcast grid bit for bit.
 */
typedef struct {
    const float* in;
    long nx, ny, nz;
    const long* bins;
    long q0, q1;
    const cplx *wx, *wy, *wz;
    double* out;
} bins_job;

static void* bins_worker(void* arg) {
    bins_job* J = (bins_job*)arg;
    for (long q = J->q0; q < J->q1; ++q) {
        long kx = J->bins[3 * q], ky = J->bins[3 * q + 1], kz = J->bins[3 * q + 2];
        double sr = 0.0, si = 0.0;
        for (long z = 0; z < J->nz; ++z) {
            cplx ez = J->wz[(kz * z) % J->nz];
            for (long y = 0; y < J->ny; ++y) {
                cplx eyz = cmul(J->wy[(ky * y) % J->ny], ez);
                const float* row = J->in + 2 * (z * J->ny + y) * J->nx;
                long ix = 0; /* (kx * x) mod nx, advanced by kx per step */
                for (long x = 0; x < J->nx; ++x) {
                    cplx a = {(double)row[2 * x], (double)row[2 * x + 1]};
                    cplx v = cmul(a, cmul(J->wx[ix], eyz));
                    sr += v.re;
                    si += v.im;
                    ix += kx;
                    if (ix >= J->nx) ix -= J->nx;
                }
            }
        }
        J->out[2 * q] = sr;
        J->out[2 * q + 1] = si;
    }
    return NULL;
}

int oracle_dft3d_bins_c64(const float* in, long nx, long ny, long nz, const long* bins, long nbins, int sign,
                          double* out, int nthreads) {
    for (long q = 0; q < nbins; ++q)
        if (bins[3 * q] < 0 || bins[3 * q] >= nx) return -1; /* the running index needs 0 <= kx < nx */
    cplx* wx = make_table(nx, sign);
    cplx* wy = make_table(ny, sign);
    cplx* wz = make_table(nz, sign);
    int rc = 0;
    if (!wx || !wy || !wz) rc = -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > nbins) nthreads = (int)(nbins > 0 ? nbins : 1);
    pthread_t th[256];
    bins_job jobs[256];
    int started = 0;
    for (int t = 0; t < nthreads && rc == 0; ++t) {
        bins_job J = {in, nx, ny, nz, bins, nbins * t / nthreads, nbins * (t + 1) / nthreads, wx, wy, wz, out};
        jobs[t] = J;
        if (pthread_create(&th[t], NULL, bins_worker, &jobs[t]) != 0) {
            rc = -1;
            break;
        }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(wx);
    free(wy);
    free(wz);
    return rc;
}

/* Library self-identification, so a loader can check it opened the oracle. */
const char* oracle_name(void) { return "gbfft FP64 oracle (test infrastructure)"; }
