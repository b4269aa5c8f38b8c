"""FP64 CPU oracle for GMF-FLBM on D3Q27 (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product library never links or
calls it; it shares no code, header or table with the CUDA path.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):

* ``tables``            pinned: Table II printed b_k, orthogonality, n_k/mu_k relation
* ``philox4x32_10``     pinned: published known-answer vectors (Salmon et al. SC'11),
                        and cuRAND's Philox4_32_10 on 202 counters/keys (GPU test)
* ``normals``           pinned: moments of the normal stream; Box-Muller identity
* ``feq2``              pinned: moments 0/1/2 exact, zero ghost projection
* ``noise_term``        pinned: conservation, single-node AR(1) stationary variance
* ``collide_node/step`` pinned: conservation, AR(1) lag-1 = 1-omega / 0, shear-wave
                        viscosity, tau=1 GMF == BGK, kT=0 cube-rotation covariance,
                        uniform-flow equilibrium fixed point at every tau and the
                        post-collision second and ghost moments of a moving state
                        (the f^eq subtraction of Eq. moments2)
* ``REG`` scheme        follows a reading (the paper does not define Reg-FLBM's
                        ghost non-equilibrium treatment: full-order Maxwellian
                        coefficients, unit ghost relaxation); the implementation of
                        that reading is pinned: tau = 1 map to the product-form
                        D3Q27 equilibrium, kT = 0 ghost coefficients rho u^deg and
                        relaxed second moment at tau = 0.6, 2, the uniform-flow
                        fixed point, and the AR(1) ghost statistics
* ``structure_factor``  pinned: numpy FFT, Parseval, single-plane-wave shell
* ``mlp`` (learned collision): forward/backward pinned by central finite
                        differences and closed forms, the projection by the
                        conservation identities, the training target by the
                        closed-form ghost synthesis; the target inherits the
                        Reg-FLBM reading (not checkable against the paper's text)
"""
from .oracle import *  # noqa: F401,F403
