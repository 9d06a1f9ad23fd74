"""Plain FP64 CPU oracle for the VOLDOR+ dense-indirect EM (test infrastructure).

This package is TEST INFRASTRUCTURE ONLY.  It defines, slowly and plainly, what
the CUDA library computes, so the library can be checked against it.  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the library never calls it and has no CPU fallback.

It shares no code with the CUDA path.  Both sides consume inputs from the
``synth`` package (which holds no estimation arithmetic).

Modules and the passage each follows (Min & Dunn, "VOLDOR+SLAM", 2021):
  philox   -- Philox4x32-10 counter RNG (Salmon et al., SC'11), the source of
              every random draw (hypotheses, P3P samples, initial depth).
  fisk     -- Fisk (log-logistic) end-point-error model and the maximum-inlier
              energy (Sec. III-A "VOLDOR+", Eq. 4 form).
  geometry -- pinhole projection, bilinear flow sampling, SE(3) exp/log.
  depth    -- depth M-step: hypothesis sampling, per-pixel argmin (Eq. 5) and
              propagation along alternately directed 1-D chains (Sec. III-A
              "Hierarchical Propagation Scheme").
  hmm      -- rigidness E-step: two-state forward-backward on chains, and the
              depth confidence map (Eq. 6).
  p3p      -- minimal 3-point pose solver (Grunert's distance formulation via
              a resultant; the paper cites AP3P, any exact P3P has the same
              solution set).
  pose     -- pose M-step: Monte-Carlo P3P sampling, dense scoring, mean-shift
              in se(3) (Eq. 7).
  eightpoint -- monocular bootstrap (8-point essential matrix on X_1).
  em       -- the iteration schedule tying the steps together.
  cnn      -- the learned initialiser (no counterpart in the paper): a small
              3x3 convolutional network from the flows to an initial inverse
              depth and rigidness, its backward pass, loss and Adam step.
  posecov  -- the pose covariance from the P3P samples: iterative Gaussian
              fit with 3-sigma rejection and an eigenvalue floor (Sec. III-A
              "Uncertainty-aware Pose Estimation").
  ka       -- keyframe alignment (Sec. III-C, Eq. 9-12): point-to-plane
              registration of two depth maps in inverse-depth form with a
              Cauchy kernel, Levenberg-Marquardt, covariance (J^T J)^-1.
  vc       -- visibility, coverage and their harmonic mean (Eq. 8), the VO
              stride and keyframe test (Sec. III-B "VO Stride and Keyframe
              Selection").
"""
