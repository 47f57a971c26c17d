"""FP64 CPU oracle for dynamic compressive spectral clustering.

Martin, Loukas, Vandergheynst, "Fast Approximate Spectral Clustering for
Dynamic Networks" (ICML 2017, arXiv:1706.03591).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method in float64 with numpy/scipy.  It exists to check the
CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product path (the CUDA library and its
Python binding) never does, and this package imports nothing from it.

Modules
-------
laplacian   normalized Laplacian and its shifted form L~ = L - I (Section 2.1)
chebyshev   Jackson-damped Chebyshev low-pass: coefficients, three-term
            recursion, moments, eigencount and the lambda_k dichotomy
            (Sections 2.2, 3.3 and 4.1)
philox      Philox-4x32-10 counter-based generator and Box-Muller normals
            (the random signal block R of Section 2.2)
kmeans      Lloyd k-means, the paper's cost C_X (Eq. 1) and brute force
spectral    exact spectral clustering by dense eigendecomposition (Section 2.1)
dynamic     Algorithm 1 (dynamic CSC) driver with the feature splice (Eq. 6)
compressive compressive k-means: variable-density sampling, reduced k-means,
            Tikhonov interpolation by k low-pass filterings (Section 2.2, step 2)
grad        gradients of a feature-space loss through the filter (coefficients
            and edge weights; the paper has no derivative)
similarity  edge similarity ||L_t - L_{t-1}||_F and Corollary 4.2's bound
            (Definition 4.1, Section 4)

Parity status of every function is stated in its module header.  The
eigencount also has the alternative trace estimator (chebyshev.trace_count).
"""
from . import laplacian, chebyshev, philox, kmeans, spectral, dynamic  # noqa: F401
from . import compressive, grad, similarity  # noqa: F401
