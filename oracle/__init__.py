"""FP64 CPU oracle for the Fourier-domain digital shearlet transform.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library; the two
meet only through arrays produced by the seeded generators.

Modules
-------
transform
    The shearlet decomposition / reconstruction / adjoint written exactly as
    the paper states them (Alg. "Shearlet Decomposition", Alg. "Shearlet
    reconstruction", the tensor listings of Sec. 3.4 and the Fourier-shift
    convention of Sec. 3.3), plus a natural-order form and a brute-force
    spatial correlation used to pin it.
bank
    The digital shearlet filter bank of Sec. 2.1 / 3.4 (1D maximally flat
    low-pass h, mirror high-pass g, iterated filters h_j, g_j, McClellan fan
    filter P, digital shear S^d of Eqs. 2.4-2.5, cones, RMS and dual frame
    weights).
apps
    Hard thresholding, PSNR, denoising (Sec. 4.2) and iterative hard
    thresholding inpainting (Alg. "Shearlet inpainting by iterative hard
    thresholding", Sec. 4.3).
nn
    The learned parts in float64 torch CPU ops: 3 x 3 convolution, PReLU,
    pools, linear, softplus, the relaxed threshold, MSE, Adam, both networks,
    the unrolled iteration (gradients by autograd).
ray
    The discrete parallel-beam ray transform of Sec. 4.4 (Joseph's method) as
    an explicit sparse matrix, and exact line integrals of ellipses.
lpd
    The learned primal-dual reconstruction of Sec. 4.4 (Algorithm 2) in the
    image and the shearlet domain.

Every function computes in float64 / complex128.
"""
