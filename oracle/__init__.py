"""FP64 CPU oracle for the semi-analytical isogeometric thermal method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The GPU
library never calls it, shares no code with it and has no CPU fallback.

Every function restates a step of the paper's method in plain numpy/scipy,
double precision, in the paper's order and notation:

* ``bspline``      Cox-de Boor B-spline basis (Section 2.3, basis of order p)
* ``geometry``     NURBS map, Jacobian, element and face quadrature (Section 2.3)
* ``assembly``     M, K and the boundary weight matrices (Section 2.3,
                   the M_ij, K_ij, F_i integrals)
* ``sources``      scan -> discrete point sources (Section 2, t^(I+1) = t^(I) + dt,
                   spacing v*dt, E = A*P*dt)
* ``pointsource``  the point-source temperature and gradient
                   (Eqs. sum-of-point-temp and semi-temperature)
* ``solver``       boundary data (Eqs. that-bc-n, that-bc-d), theta-scheme
                   (Eq. theta-method) and reconstruction T = T~ + T^

Readings of the paper where it is silent or ambiguous (all also recorded in
the design notes):
  R1 source I (1-based) sits at arc length (I-1)*v*dt along its track and is
     active from step I on (t^(I) = I*dt); its age at step n is
     (n-I)*dt + r^2/(8*alpha).
  R2 half-space factor s_img = 2 by default (image source across the adiabatic
     top plane); s_img = 1 reproduces the printed full-space kernel.
  R3 sources sit on the planar top face z = z_top.
  R4 (p+1) Gauss-Legendre points per direction per element and per face
     element.
  R5 bottom control variables are set to the L2 projection of T_c - T~ onto
     the bottom-face spline space.
"""
