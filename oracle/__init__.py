"""FP64 CPU oracle for the Fourier-domain Log-SP decoder (Kasai & Sakaniwa, IEICE 2010).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or link this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it. It shares no code with the CUDA path
(``paper_1008_4370_gb300``): it builds its own GF(2^m) tables, its own Fourier index
maps and its own graph adjacency from the plain edge list.

Two independent decoders are written out here, both in float64 and in the paper's own
order of steps:

* ``sp``          -- probability-domain sum-product (Section 2.1, Eq. (1) of the check-node
                     update, the XOR convolution computed from its definition, O(q^2)).
* ``logfourier``  -- the Log-Fourier SP decoder (Section 3.2): WHT + Gamma initialisation,
                     permuted leave-one-out sums at the check nodes, the signed log-convolution
                     of the boxplus definition at the variable nodes, bit decisions and
                     syndrome bits read from the Fourier domain.

``bruteforce`` enumerates codewords of tiny codes for exact symbol-MAP / bit-MAP marginals.

Pins (tests/test_oracle_*.py) tie every function to something other than itself:
the GF(8) table and the z.x = 3 example printed in Section 2/2.1, the companion-matrix
identity of Appendix A, the Fourier permutation identity proved in Appendix A, W.W = qI,
Parseval, the tanh closed form of the channel message, the Gamma homomorphism, equality of
the two decoders' messages, and brute-force MAP on cycle-free graphs.
Parity status: every public function is pinned; see the per-module headers.
"""

from . import gf, transforms, channel, code, sp, logfourier, bruteforce  # noqa: F401
