"""Rasterizer constants and conventions.

The paper (Sec. 3.1, "Review of Gaussian-Splatting", Eq. alpha-blending; Sec. A)
uses the unmodified 3DGS tile rasterizer and states none of its constants. This
oracle and the CUDA library both adopt the values below; they are a reading of
the paper, not something it pins, so no test can pin them against the paper.

  TILE        16 x 16 pixel tiles
  DILATION    0.3 px^2 added to both diagonal entries of the 2D covariance
  NEAR        a Gaussian is visible only if its camera-space depth tz > 0.2
  RADIUS_SIG  splat radius = ceil(3 * sqrt(largest eigenvalue of the 2D covariance))
  ALPHA_MAX   alpha = min(0.99, opacity * G)
  ALPHA_MIN   a splat with alpha < 1/255 is skipped at that pixel
  T_MIN       walking front to back, stop before the splat that would bring T below 1e-4
  SH_OFFSET   colour = max(0, SH(dir) + 0.5) per channel
  background  black
  pixel centre (px + 0.5, py + 0.5); tile rect of a splat covers the tiles
              floor((mu - r)/16) .. floor((mu + r)/16) on each axis, clipped to the image
  order       splats of a tile are blended by (float32 depth, Gaussian index) ascending
  smooth mode (test only): no alpha clamp, no alpha skip, no T stop, no SH clamp and
              every visible splat is blended at every pixel
"""
TILE = 16
DILATION = 0.3
NEAR = 0.2
RADIUS_SIG = 3.0
ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4
SH_OFFSET = 0.5
