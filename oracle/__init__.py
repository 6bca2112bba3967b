"""CPU oracle of the vectorized Sparrow step and of the Q-network.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2305_04180_gb300``) never imports it and
it imports nothing of the product path.

* ``sparrow_oracle.c`` -- the environment step in plain C, built twice:
  strict float32 (``f32``, the precision of the paper's torch world matrix)
  and float64 (``f64``, libm transcendental functions).
* ``qnet.py`` -- the dueling MLP Q-network, TD loss, gradients and Adam in
  float64 numpy.

Parity status: every oracle function is pinned by the ``-m "not gpu"`` tests
(closed forms, brute force, analytic geometry, finite differences); none is
"parity unpinned".
"""

from .sim import OracleSim, build_oracle, lib, pack_map, rng_u64

__all__ = ["OracleSim", "build_oracle", "lib", "pack_map", "rng_u64"]
