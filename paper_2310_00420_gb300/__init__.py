"""GB300-native covariance-free EM for clustered multi-task compressive sensing.

The compute path lives in ``libcmcs.so`` (CUDA for sm_103a, C ABI declared in
``include/cmcs.h``); ``cmcs`` is its thin ctypes binding and ``synth`` the seeded synthetic
workload generator.  Importing this package loads nothing native; the binding loads the
library on first use and raises if it is missing.

Typical use (device tensors or host arrays; Phi is [sum_t N_t][D] row-major)::

    from paper_2310_00420_gb300 import cmcs
    with cmcs.Context(Phi, y, N, C=4, K=32, beta=1e4, precision="bf16x3",
                      refine_max=8, refine_tol=1e-5) as ctx:
        ctx.em_iter(50)                       # Alg. 2: E-step (Sec. 3) + M-step (Eq. 5)
        mu = ctx.read(cmcs.OUT_MU)            # [T][C][D] posterior means of the last E-step
        q = ctx.read(cmcs.OUT_Q)              # [T][C] responsibilities
        a = ctx.read(cmcs.OUT_ASSIGN)         # [T] cluster assignments
        z = ctx.read(cmcs.OUT_RECON)          # [T][D] reconstructions mu_{t, a_t}

``cmcs.Context(None, y, N, mask=mask, ...)`` (or ``Context.from_fourier``) takes the
structured sensing matrices of Sec. 4, Phi_t = Omega_t F, given by their frequency masks.
Keyword switches select the method's variants (``learn_pi``, ``probe_share``, ``precond``,
``warm_start``); ``Context.adjoint`` and ``adjoint.posterior_means`` (a torch autograd
Function) differentiate the means.
"""
