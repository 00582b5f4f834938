/*
 * Allen-Cahn oracle: plain, slow, FP64 CPU restatement of the explicit
 * finite-difference scheme of Kim, "Fast Numerical Simulation of Allen-Cahn
 * Equation" (arXiv 2105.09671).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library) shares no code, header, table or helper with it.
 *
 * Every routine follows the paper's notation and order of operations:
 *   - Section 2: cell-centred grid x_i = a + (i - 0.5) h, extended by one
 *     ghost layer per side; zero-Neumann boundary by copying the adjacent
 *     interior value into the ghost; dt = 0.1 h^2 is chosen by the caller.
 *   - Eq. (pytorchACeq), Section 2.1: phi^{n+1} = phi^n
 *       + dt * ((phi^n - (phi^n)^3) / eps^2 + Lap_h phi^n),
 *     Lap_h phi = (phi_{i-1,j} + phi_{i+1,j} + phi_{i,j-1} + phi_{i,j+1}
 *                  - 4 phi_{ij}) / h^2     (7-point analogue in 3D).
 *   - Section 3.1: circle/sphere tanh initial conditions and the random
 *     initial condition 0.1 * rand with rand in [-1, 1).
 *   - The discrete Ginzburg-Landau energy and the phase volume are not in
 *     the paper; they are the plain definitions written out (see the
 *     comments at each routine).
 *
 * Readings of the paper that this file takes:
 *   - The neighbour sum is evaluated in the paired order (W + E) + (S + N)
 *     [+ (B + F)], so that grid mirror and transpose symmetries hold bit for
 *     bit; in exact arithmetic every order is the same.
 *   - The ghost faces cover the interior range of the other indices; corner
 *     and edge ghosts are never read by the 5/7-point stencil.
 *   - The random draw is SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as
 *     a counter-based generator: cell with linear index c under seed s takes
 *     output number c + 1 of the SplitMix64 sequence whose state starts at s.
 *     rand = 2 * (z >> 11) * 2^-53 - 1, phi0 = 0.1 * rand.
 *
 * Build: gcc -O2 -ffp-contract=off (no FMA contraction), optional OpenMP
 * over rows / planes (each cell is computed independently, so the result is
 * the same for every thread count).  Reductions are serial in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EXPORT __attribute__((visibility("default")))

/* ---------------------------------------------------------------- 2D ---- */

/* Index into the extended (Nx+2) x (Ny+2) array of Section 2, 0-based:
 * extended column I = 0..Nx+1, row J = 0..Ny+1; interior is 1..Nx, 1..Ny. */
#define EXT2(I, J) ((size_t)(J) * (size_t)(nx + 2) + (size_t)(I))

/* Zero-Neumann boundary of Section 2: each ghost copies its interior
 * neighbour.  The bottom/top faces run over the interior columns, the
 * left/right faces over the interior rows. */
static void fill_ghosts2d(int64_t nx, int64_t ny, double *e) {
  for (int64_t i = 1; i <= nx; ++i) {
    e[EXT2(i, 0)] = e[EXT2(i, 1)];
    e[EXT2(i, ny + 1)] = e[EXT2(i, ny)];
  }
  for (int64_t j = 1; j <= ny; ++j) {
    e[EXT2(0, j)] = e[EXT2(1, j)];
    e[EXT2(nx + 1, j)] = e[EXT2(nx, j)];
  }
}

/* nsteps explicit Euler steps of Eq. (pytorchACeq) on an nx-by-ny grid.
 * phi_in / phi_out: row-major [ny][nx] FP64 (x fastest); they may alias.
 * Returns 0, or -1 on bad arguments / allocation failure. */
EXPORT int oracle_step2d(int64_t nx, int64_t ny, double h, double eps, double dt,
                         const double *phi_in, double *phi_out, int64_t nsteps) {
  if (nx < 1 || ny < 1 || nsteps < 0 || !(h > 0) || !(eps > 0) || !(dt >= 0))
    return -1;
  size_t ext = (size_t)(nx + 2) * (size_t)(ny + 2);
  double *a = (double *)calloc(ext, sizeof(double));
  double *b = (double *)calloc(ext, sizeof(double));
  if (!a || !b) { free(a); free(b); return -1; }
  for (int64_t j = 0; j < ny; ++j)
    for (int64_t i = 0; i < nx; ++i)
      a[EXT2(i + 1, j + 1)] = phi_in[(size_t)j * nx + i];
  const double eps2 = eps * eps, h2 = h * h;
  for (int64_t n = 0; n < nsteps; ++n) {
    fill_ghosts2d(nx, ny, a);
#pragma omp parallel for schedule(static)
    for (int64_t j = 1; j <= ny; ++j) {
      for (int64_t i = 1; i <= nx; ++i) {
        double p = a[EXT2(i, j)];
        double w = a[EXT2(i - 1, j)], e = a[EXT2(i + 1, j)];
        double s = a[EXT2(i, j - 1)], nn = a[EXT2(i, j + 1)];
        double lap = ((w + e) + (s + nn) - 4.0 * p) / h2;
        double reaction = (p - p * p * p) / eps2;
        b[EXT2(i, j)] = p + dt * (reaction + lap);
      }
    }
    double *t = a; a = b; b = t;
  }
  for (int64_t j = 0; j < ny; ++j)
    for (int64_t i = 0; i < nx; ++i)
      phi_out[(size_t)j * nx + i] = a[EXT2(i + 1, j + 1)];
  free(a); free(b);
  return 0;
}

/* ---------------------------------------------------------------- 3D ---- */

#define EXT3(I, J, K) \
  (((size_t)(K) * (size_t)(ny + 2) + (size_t)(J)) * (size_t)(nx + 2) + (size_t)(I))

static void fill_ghosts3d(int64_t nx, int64_t ny, int64_t nz, double *e) {
  for (int64_t k = 1; k <= nz; ++k)
    for (int64_t j = 1; j <= ny; ++j) {
      e[EXT3(0, j, k)] = e[EXT3(1, j, k)];
      e[EXT3(nx + 1, j, k)] = e[EXT3(nx, j, k)];
    }
  for (int64_t k = 1; k <= nz; ++k)
    for (int64_t i = 1; i <= nx; ++i) {
      e[EXT3(i, 0, k)] = e[EXT3(i, 1, k)];
      e[EXT3(i, ny + 1, k)] = e[EXT3(i, ny, k)];
    }
  for (int64_t j = 1; j <= ny; ++j)
    for (int64_t i = 1; i <= nx; ++i) {
      e[EXT3(i, j, 0)] = e[EXT3(i, j, 1)];
      e[EXT3(i, j, nz + 1)] = e[EXT3(i, j, nz)];
    }
}

/* 3D extension of Eq. (pytorchACeq) with the 7-point Laplacian
 * (Section 2 states the 3D scheme extends the 2D one; Section 2.2 uses the
 * 3D replication pad and a 3D second-difference filter).
 * phi: [nz][ny][nx] FP64, x fastest. */
EXPORT int oracle_step3d(int64_t nx, int64_t ny, int64_t nz, double h, double eps,
                         double dt, const double *phi_in, double *phi_out,
                         int64_t nsteps) {
  if (nx < 1 || ny < 1 || nz < 1 || nsteps < 0 || !(h > 0) || !(eps > 0) ||
      !(dt >= 0))
    return -1;
  size_t ext = (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
  double *a = (double *)calloc(ext, sizeof(double));
  double *b = (double *)calloc(ext, sizeof(double));
  if (!a || !b) { free(a); free(b); return -1; }
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i)
        a[EXT3(i + 1, j + 1, k + 1)] = phi_in[((size_t)k * ny + j) * nx + i];
  const double eps2 = eps * eps, h2 = h * h;
  for (int64_t n = 0; n < nsteps; ++n) {
    fill_ghosts3d(nx, ny, nz, a);
#pragma omp parallel for schedule(static)
    for (int64_t k = 1; k <= nz; ++k) {
      for (int64_t j = 1; j <= ny; ++j) {
        for (int64_t i = 1; i <= nx; ++i) {
          double p = a[EXT3(i, j, k)];
          double w = a[EXT3(i - 1, j, k)], e = a[EXT3(i + 1, j, k)];
          double s = a[EXT3(i, j - 1, k)], nn = a[EXT3(i, j + 1, k)];
          double bo = a[EXT3(i, j, k - 1)], f = a[EXT3(i, j, k + 1)];
          double lap = ((w + e) + (s + nn) + (bo + f) - 6.0 * p) / h2;
          double reaction = (p - p * p * p) / eps2;
          b[EXT3(i, j, k)] = p + dt * (reaction + lap);
        }
      }
    }
    double *t = a; a = b; b = t;
  }
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i)
        phi_out[((size_t)k * ny + j) * nx + i] = a[EXT3(i + 1, j + 1, k + 1)];
  free(a); free(b);
  return 0;
}

/* ------------------------------------------------- initial conditions ---- */

/* Circle (2D, nz == 1) or sphere (3D) of Section 3.1:
 *   phi0 = tanh((R0 - |x - c|) / (sqrt(2) eps)),
 * cell centres x_i = a + (i - 0.5) h for i = 1..N (Section 2), so with
 * 0-based index i the centre is a + (i + 0.5) h.  (ax, ay, az) is the lower
 * domain corner (a, c[, e]); c = (cx, cy, cz). */
EXPORT void oracle_init_sphere(int64_t nx, int64_t ny, int64_t nz, double h,
                               double ax, double ay, double az, double cx,
                               double cy, double cz, double r0, double eps,
                               double *phi) {
  const double w = sqrt(2.0) * eps;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        double x = ax + ((double)i + 0.5) * h;
        double y = ay + ((double)j + 0.5) * h;
        double dx = x - cx, dy = y - cy;
        double r2 = dx * dx + dy * dy;
        if (nz > 1) {
          double z = az + ((double)k + 0.5) * h;
          double dz = z - cz;
          r2 += dz * dz;
        }
        phi[((size_t)k * ny + j) * nx + i] = tanh((r0 - sqrt(r2)) / w);
      }
}

/* SplitMix64 output number (counter + 1) of the sequence seeded with
 * `seed` (Steele, Lea, Flood 2014): the state advances by the golden-gamma
 * 0x9E3779B97F4A7C15 and each output is the state passed through the
 * variant-13 finaliser. */
EXPORT uint64_t oracle_splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Random initial condition of Section 3.1: phi0 = 0.1 * rand, rand uniform
 * in [-1, 1), cell c = linear index (x fastest) of an n-cell grid. */
EXPORT void oracle_init_random(int64_t n, uint64_t seed, double amplitude,
                               double *phi) {
  for (int64_t c = 0; c < n; ++c) {
    uint64_t z = oracle_splitmix64(seed, (uint64_t)c);
    double u = (double)(z >> 11) * 0x1.0p-53; /* [0, 1), exact */
    double r = 2.0 * u - 1.0;                 /* [-1, 1), exact */
    phi[c] = amplitude * r;
  }
}

/* ------------------------------------------------------ reductions ------ */

/* Discrete Ginzburg-Landau energy whose gradient flow is the scheme:
 *   E_h = h^d [ sum_cells F(phi)/eps^2
 *              + 1/2 sum_{interior faces (a,b)} ((phi_a - phi_b)/h)^2 ],
 * F(phi) = 0.25 (phi^2 - 1)^2 (Section 1).  Boundary faces carry zero
 * difference under the zero-Neumann ghosts, so only interior faces count.
 * dE_h/dphi_c = -h^d * RHS_c, with RHS the bracket of Eq. (pytorchACeq).
 * Serial FP64 sum in index order; nz == 1 means 2D. */
EXPORT double oracle_energy(int64_t nx, int64_t ny, int64_t nz, double h,
                            double eps, const double *phi) {
  const int d = nz > 1 ? 3 : 2;
  double bulk = 0.0, grad = 0.0;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        size_t c = ((size_t)k * ny + j) * nx + i;
        double p = phi[c];
        double q = p * p - 1.0;
        bulk += 0.25 * q * q;
        if (i + 1 < nx) { double g = (phi[c + 1] - p) / h; grad += g * g; }
        if (j + 1 < ny) { double g = (phi[c + nx] - p) / h; grad += g * g; }
        if (k + 1 < nz) {
          double g = (phi[c + (size_t)nx * ny] - p) / h; grad += g * g;
        }
      }
  double hd = d == 3 ? h * h * h : h * h;
  return hd * (bulk / (eps * eps) + 0.5 * grad);
}

/* Phase volume of {phi > 0} in the diffuse sense: V = h^d sum (1 + phi)/2.
 * The equivalent radius is sqrt(V/pi) in 2D and (3V/(4 pi))^(1/3) in 3D,
 * compared with the shrinking law r(t)^2 = r0^2 + 2(1 - d) t of Section 3.2. */
EXPORT double oracle_phase_volume(int64_t nx, int64_t ny, int64_t nz, double h,
                                  const double *phi) {
  const int d = nz > 1 ? 3 : 2;
  double s = 0.0;
  size_t n = (size_t)nx * ny * nz;
  for (size_t c = 0; c < n; ++c) s += 0.5 * (1.0 + phi[c]);
  double hd = d == 3 ? h * h * h : h * h;
  return hd * s;
}

/* Threads of the following OpenMP loops (n <= 0 restores the default). */
EXPORT void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
  (void)n;
#endif
}

/* Number of OpenMP threads the stepping loops use (1 without OpenMP). */
EXPORT int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
