"""CPU reference ("oracle") for the time-spectral GLS Navier-Stokes operator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its Python binding) never calls it, and this
package never imports the product.

It is a plain, slow, FP64 restatement of Esmaily & Jia, "A new stabilized
time-spectral finite element solver for fast simulation of blood flow"
(arXiv 2311.09465), in the paper's own representation:

* full complex mode vectors of length 2N-1 (modes -N+1..N-1), section 2.1,
  eq. (phi-def);
* the explicit truncated convolution matrix A_{mn} = u_{m-n}, |m-n| < N,
  eq. (phi-def) -- not time sampling;
* tau = [A_i G_ij A_j + C_I kappa^2 G_ij G_ij I]^{-1/2} through a library
  Hermitian eigensolver, eq. (3D-tau) and the remark that follows it;
* element-order accumulation of the discrete residual, eq. (Rmc), and of the
  tangent blocks, eq. (K_mat), with no colouring.

Modules:
  spectral   mode vectors, convolution matrix, Omega (eq. phi-def)
  geometry   P1 tetrahedron gradients, metric G (eq. metric), quadrature
  tau        stabilisation matrix (eq. 3D-tau)
  operator   residual (eq. Rmc) and Jacobian-vector products (eq. K_mat)
  assemble   dense tangent H from eq. (K_mat) block by block (small meshes)
  steady     independent steady SUPG/PSPG residual (eq. NSt-weak, omega = 0)
  solver     restarted GMRES, dense LU, pseudo-time Newton (sections 2.4-2.5)
  precond    nodal block Jacobi and symmetric block Gauss-Seidel on nodal blocks
  womersley  closed-form pulsatile pipe flow with its own Bessel series

Parity status of each function is stated in its module docstring.
"""
