"""FP64 CPU oracle for the Neural Shadow Mapping hot path.

TEST INFRASTRUCTURE.  This package is the plain, slow, obviously correct
statement of what the GPU path computes; it exists to check that path.  Only
the test-suite, the smoke check of the package entry file and the CPU-baseline
leg of the benchmark may import it.  The product library never imports,
links or executes anything here, and nothing here imports the product.

Contents
  gather   -- texel lookup and hard depth test (binary32-exact definition),
              the four input features (Sec. 3.1, 3.2, Fig. 2), the blocker
              search and the penumbra-width model (Sec. 3.6, suppl. Sec. 4).
  network  -- the compact encoder/decoder (Sec. 3.5), its adjoint, the
              Eq. 2 loss (L1 part) and an Adam step.
  temporal -- the temporal-instability metric (Sec. 3.4, Eq. 3) and the
              penumbra-size histogram / 95th percentile / depth rule (Sec. 3.6).
  train_weights -- a script that trains seeded weights with the functions
              above (an input for the tests and the benchmark, never an
              expected value).

Pinning status (what checks each function against something other than
itself; the tests under tests/test_oracle_*.py):
  project_fp32 / lookup_and_test -- brute-force shadow rays on tiny scenes,
      the sphere-over-plane shadow conic, hand-built projections with known
      texel indices, the FP64 index (differences only at texel boundaries).
  features -- closed forms on hand-built pixels; invariants on rendered frames.
  blocker_search -- brute force over the whole map on tiny inputs, the
      no-occluder and k = 0 special cases.
  blocker_window_half -- the emitter radius carried to the receiver's depth
      and projected through the light's own view-projection matrix, in
      texels, over several light distances (fov) and map widths; a
      hand-worked case that a Ws-for-Ws/2, tan(fov)-for-tan(fov/2) or
      diameter-for-radius error would change.
  penumbra_width -- the r_e = 0 and r_s = 0 closed forms (similar triangles).
  conv2d / avgpool2 / upsample2 -- direct summation loops, torch FP64
      library routines, adjoint dot-product identities.
  forward / backward -- forward against the network written out level by
      level with direct-summation convolutions, explicit 2 x 2 means and loop
      bilinear up-sampling (3 and 4 levels, 8 x 8 inputs: a dropped skip, a
      missing ReLU or pooling before the ReLU each fail it); backward against
      central finite differences; parameter and MAC counts against the
      paper's printed table values.  The paper prints no worked example of
      the network's output; trained weights are only inputs to these
      definitions.
  loss_l1 / adam_update / train_step -- closed forms on small vectors and
      finite differences of the loss.
  reproject_fp32 / accept_fp32 / instability_pair / temporal_instability --
      rays through pixel centres reproject to their pixel; identical frames
      give 0; a constant difference gives the closed form; depth, normal and
      coverage rejections by construction; with a moved camera the
      reprojection finds the same surface point within about a pixel.
  screen_width_px / penumbra_histogram / p95_from_histogram / depth_for_width
      -- projected endpoints, hand histograms, the uniform distribution's
      percentile, and the paper's 24 / 96 / 384-pixel receptive fields of the
      3 / 5 / 7-level nets.
  space_to_depth / s2d_output / forward_s2d (Sec. 3.5, the space-to-depth
      topology) -- the index map by brute force, the detail placement and
      channel-0 bilinear by explicit loops, the whole network against a
      direct-summation loop implementation on 8 x 8 inputs, and the head-bias
      closed form.
  backward_s2d / train_step_s2d -- the dot-product identity of the two new
      operator adjoints, central differences on weights and features, the
      training step against its parts.
  round_bf16 / round_bf16_pair / round_e4m3 -- the formats' bit fields
      (enumerated value sets, ties to even, saturation).
  round_e4m3_terms / round_e4m3_terms_per_out_channel -- one term equals
      round_e4m3; E4M3 values reproduce exactly and a quarter-ulp offset needs
      the second term; the three-term error bound (2^-12 relative plus a
      subnormal floor) over random values; saturation at 448 + 28 + 1.75.
"""
