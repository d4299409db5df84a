"""Plain FP64 CPU oracle for s-FairSC — TEST INFRASTRUCTURE, not the product.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import anything from this package.  The library path never calls it; it
shares no code with the CUDA kernels (the only shared module is `msbm`, the
seeded graph generator, which holds none of the method's arithmetic).

Everything follows Wang, Lu, Davidson and Bai, "Scalable Spectral Clustering
with Group Fairness Constraints" (AISTATS 2023):

  problem.py   graph Laplacian, normalized Laplacian, G, F0, F, C, sigma
               (Sec. 2.1 eq. group-vec / f0h, Lemma 2.1, Sec. 3.2, App. C)
  fairsc.py    dense FairSC (Algorithm 2), the first variant (eq. lveig) and
               the dense s-FairSC matrix (eq. asigma)
  sfairsc.py   the matrix-free operator of Sec. 3.4 (i)-(ii) and Algorithm 3
  lanczos.py   a plain thick-restart Lanczos used for sizes where a dense
               eigendecomposition does not fit
  kmeans.py    seeded k-means++ / Lloyd (Algorithm 3 step 4)
  metrics.py   error rate (eq. err) and balance (eq. bal, eq. avebal)
  gradient.py  d(sum of the k smallest eigenvalues)/d(edge weight, bandwidth)

Parity pins for every function live in tests/ (markers "not gpu").
"""
