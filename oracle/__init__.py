"""Plain CPU FP64 oracle of the PWL current-based VIE (arXiv 1902.02196).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the CPU-baseline leg of the benchmark may import anything from here.  The
product path (the CUDA library and its Python binding) never calls it, and
this package never imports the product package: the two share no code.  The
only common module is `synth`, which generates seeded inputs and holds none of
the method's arithmetic.

Everything here is written for a reader who checks it against the paper:
  * green.py     -- Galerkin entries of the N operator (Section III-C, Eq. 25,
                    Eq. 34) by a reduction of the singular 6-D integrals to 3-D
                    and 2-D integrals of g times polynomials, evaluated with
                    Gauss-Legendre and Duffy-Gauss rules; Gram tensor (Eq. 33).
  * operator.py  -- dense MoM matrix A = M_eps G - M_chi N (Eq. 24) for tiny
                    grids and the FFT-accelerated circulant matvec (Section IV-A).
  * solver.py    -- restarted GMRES with the preconditioner P = M_eps G
                    (Section IV-B, Eq. 17) and a dense direct solve.
  * rhs.py       -- tested incident fields (Eq. 27, Eq. 30) and right-hand side
                    (Eq. 31) for a plane wave and for Hertzian dipoles.
  * post.py      -- tested total fields divided by the Gram matrix and the
                    absorbed power (Section IV-C, Eq. 44).
  * mie.py       -- Mie series absorbed power of a homogeneous sphere.
"""

C0 = 299792458.0  # speed of light in vacuum, m/s (exact)
EPS0 = 8.8541878128e-12  # vacuum permittivity, F/m (CODATA 2018)
MU0 = 1.0 / (EPS0 * C0 * C0)  # vacuum permeability, H/m
