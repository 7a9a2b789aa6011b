"""Plain FP64 CPU oracle for the PCEXP Krylov step on DG Euler.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run anything here;
the product (the CUDA library and its Python binding) never does, and has no
CPU fallback.  The oracle shares no code with the CUDA path: it builds its
own quadrature, basis, face list, flux and Krylov machinery from the paper
("An Exponential Time-Integrator Scheme for Steady and Unsteady Inviscid
Flows", Li, Luo, Wang & Ju).  Each function cites the section or equation it
follows.  Inputs (meshes, seeds) come from the ``workloads`` module, which
holds no method arithmetic.

Pinned by the ``-m "not gpu"`` tests against closed forms, library routines
and printed values (Table 1 "timesize", Eq. grow / exp1_grow / rkgrow,
phi_1(z) = (e^z - 1)/z, dense expm, free-stream preservation, conservation,
complex-step derivatives, the Appendix flux Jacobian (also with the rotating-frame
terms of Eq. dfdu), the inscribed-circle and inscribed-sphere diameters behind the
element time step of Eq. x3d, and the exact decay of a linear system under the
steady march of Eq. cfl); ETD2 against the scalar phi_1/phi_2 closed forms, exact
affine flows and second-order convergence; the Krylov error estimate against the
true error from a dense exponential; the stretched mesh against the spacings the
paper prints; the wall force, entropy error and density norm against trapezoid,
shoelace and closed-form integrals; the exact translation of the isentropic vortex;
the rotating-frame source of a uniform state.  Parity unpinned: the nonlinear
bump-channel steady march beyond agreement with itself (no printed number exists
for it).
"""
