// Generated by gen_coeffs.py -- do not edit by hand.
// ENO-MR candidate tables (arXiv 2311.15504, Eq. Candidates, Tables 1-4),
// derived in exact rational arithmetic and rounded once to double.
#pragma once

namespace enomr {

template <int R> struct Tab;           // T = number of tested candidates
template <int R, int t> struct Cand;   // m, n of the t-th tested candidate

// ---- order 5: g = 3, window 5, 4 tested candidates
template <> struct Tab<5> { static constexpr int T = 4; };
template <> struct Cand<5, 0> { static constexpr int m = 2, n = 2; };
template <> struct Cand<5, 1> { static constexpr int m = 1, n = 2; };
template <> struct Cand<5, 2> { static constexpr int m = 2, n = 1; };
template <> struct Cand<5, 3> { static constexpr int m = 1, n = 1; };
// b_l (rows t, columns l = -(g-1)..g-1; zero outside the stencil)
static __constant__ double kB5[20] = {
    1.0, -4.0, 6.0, -4.0, 1.0,
    0.0, -1.0, 3.0, -3.0, 1.0,
    -1.0, 3.0, -3.0, 1.0, 0.0,
    0.0, 1.0, -2.0, 1.0, 0.0,
};
// a_l (same layout)
static __constant__ double kA5[20] = {
    0x1.1111111111111p-5, -0x1.bbbbbbbbbbbbcp-3, 0x1.9111111111111p-1, 0x1.ccccccccccccdp-2, -0x1.999999999999ap-5,
    0.0, -0x1.5555555555555p-4, 0x1.2aaaaaaaaaaabp-1, 0x1.2aaaaaaaaaaabp-1, -0x1.5555555555555p-4,
    0x1.5555555555555p-4, -0x1.aaaaaaaaaaaabp-2, 0x1.1555555555555p+0, 0x1.0000000000000p-2, 0.0,
    0.0, -0x1.5555555555555p-3, 0x1.aaaaaaaaaaaabp-1, 0x1.5555555555555p-2, 0.0,
};

// ---- order 7: g = 4, window 7, 7 tested candidates
template <> struct Tab<7> { static constexpr int T = 7; };
template <> struct Cand<7, 0> { static constexpr int m = 3, n = 3; };
template <> struct Cand<7, 1> { static constexpr int m = 2, n = 3; };
template <> struct Cand<7, 2> { static constexpr int m = 3, n = 2; };
template <> struct Cand<7, 3> { static constexpr int m = 2, n = 2; };
template <> struct Cand<7, 4> { static constexpr int m = 1, n = 2; };
template <> struct Cand<7, 5> { static constexpr int m = 2, n = 1; };
template <> struct Cand<7, 6> { static constexpr int m = 1, n = 1; };
// b_l (rows t, columns l = -(g-1)..g-1; zero outside the stencil)
static __constant__ double kB7[49] = {
    1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0,
    0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0,
    -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0,
    0.0, 1.0, -4.0, 6.0, -4.0, 1.0, 0.0,
    0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0,
    0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0,
    0.0, 0.0, 1.0, -2.0, 1.0, 0.0, 0.0,
};
// a_l (same layout)
static __constant__ double kA7[49] = {
    -0x1.d41d41d41d41dp-8, 0x1.e79e79e79e79ep-5, -0x1.ec7ec7ec7ec7fp-3, 0x1.84e04e04e04e0p-1, 0x1.04e04e04e04e0p-1, -0x1.7297297297297p-4, 0x1.3813813813814p-7,
    0.0, 0x1.1111111111111p-6, -0x1.1111111111111p-3, 0x1.3bbbbbbbbbbbcp-1, 0x1.3bbbbbbbbbbbcp-1, -0x1.1111111111111p-3, 0x1.1111111111111p-6,
    -0x1.1111111111111p-6, 0x1.ddddddddddddep-4, -0x1.8888888888889p-2, 0x1.e666666666666p-1, 0x1.7777777777777p-2, -0x1.1111111111111p-5, 0.0,
    0.0, 0x1.1111111111111p-5, -0x1.bbbbbbbbbbbbcp-3, 0x1.9111111111111p-1, 0x1.ccccccccccccdp-2, -0x1.999999999999ap-5, 0.0,
    0.0, 0.0, -0x1.5555555555555p-4, 0x1.2aaaaaaaaaaabp-1, 0x1.2aaaaaaaaaaabp-1, -0x1.5555555555555p-4, 0.0,
    0.0, 0x1.5555555555555p-4, -0x1.aaaaaaaaaaaabp-2, 0x1.1555555555555p+0, 0x1.0000000000000p-2, 0.0, 0.0,
    0.0, 0.0, -0x1.5555555555555p-3, 0x1.aaaaaaaaaaaabp-1, 0x1.5555555555555p-2, 0.0, 0.0,
};

// ---- order 9: g = 5, window 9, 10 tested candidates
template <> struct Tab<9> { static constexpr int T = 10; };
template <> struct Cand<9, 0> { static constexpr int m = 4, n = 4; };
template <> struct Cand<9, 1> { static constexpr int m = 3, n = 4; };
template <> struct Cand<9, 2> { static constexpr int m = 4, n = 3; };
template <> struct Cand<9, 3> { static constexpr int m = 3, n = 3; };
template <> struct Cand<9, 4> { static constexpr int m = 2, n = 3; };
template <> struct Cand<9, 5> { static constexpr int m = 3, n = 2; };
template <> struct Cand<9, 6> { static constexpr int m = 2, n = 2; };
template <> struct Cand<9, 7> { static constexpr int m = 1, n = 2; };
template <> struct Cand<9, 8> { static constexpr int m = 2, n = 1; };
template <> struct Cand<9, 9> { static constexpr int m = 1, n = 1; };
// b_l (rows t, columns l = -(g-1)..g-1; zero outside the stencil)
static __constant__ double kB9[90] = {
    1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0,
    0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0,
    -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0,
    0.0, 1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0, 0.0,
    0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0,
    0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0,
    0.0, 0.0, 1.0, -4.0, 6.0, -4.0, 1.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 1.0, -2.0, 1.0, 0.0, 0.0, 0.0,
};
// a_l (same layout)
static __constant__ double kA9[90] = {
    0x1.a01a01a01a01ap-10, -0x1.0a90a90a90a91p-6, 0x1.4374374374374p-4, -0x1.0478478478478p-2, 0x1.7dc3dc3dc3dc4p-1, 0x1.175d75d75d75dp-1, -0x1.efbefbefbefbfp-4, 0x1.6596596596596p-6, -0x1.0410410410410p-9,
    0.0, -0x1.d41d41d41d41dp-9, 0x1.1ad1ad1ad1ad2p-5, -0x1.52e52e52e52e5p-3, 0x1.44e04e04e04e0p-1, 0x1.44e04e04e04e0p-1, -0x1.52e52e52e52e5p-3, 0x1.1ad1ad1ad1ad2p-5, -0x1.d41d41d41d41dp-9,
    0x1.d41d41d41d41dp-9, -0x1.0750750750750p-5, 0x1.1381381381381p-3, -0x1.763f63f63f63fp-2, 0x1.c4e04e04e04e0p-1, 0x1.bcf3cf3cf3cf4p-2, -0x1.0c30c30c30c31p-4, 0x1.8618618618618p-8, 0.0,
    0.0, -0x1.d41d41d41d41dp-8, 0x1.e79e79e79e79ep-5, -0x1.ec7ec7ec7ec7fp-3, 0x1.84e04e04e04e0p-1, 0x1.04e04e04e04e0p-1, -0x1.7297297297297p-4, 0x1.3813813813814p-7, 0.0,
    0.0, 0.0, 0x1.1111111111111p-6, -0x1.1111111111111p-3, 0x1.3bbbbbbbbbbbcp-1, 0x1.3bbbbbbbbbbbcp-1, -0x1.1111111111111p-3, 0x1.1111111111111p-6, 0.0,
    0.0, -0x1.1111111111111p-6, 0x1.ddddddddddddep-4, -0x1.8888888888889p-2, 0x1.e666666666666p-1, 0x1.7777777777777p-2, -0x1.1111111111111p-5, 0.0, 0.0,
    0.0, 0.0, 0x1.1111111111111p-5, -0x1.bbbbbbbbbbbbcp-3, 0x1.9111111111111p-1, 0x1.ccccccccccccdp-2, -0x1.999999999999ap-5, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.5555555555555p-4, 0x1.2aaaaaaaaaaabp-1, 0x1.2aaaaaaaaaaabp-1, -0x1.5555555555555p-4, 0.0, 0.0,
    0.0, 0.0, 0x1.5555555555555p-4, -0x1.aaaaaaaaaaaabp-2, 0x1.1555555555555p+0, 0x1.0000000000000p-2, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.5555555555555p-3, 0x1.aaaaaaaaaaaabp-1, 0x1.5555555555555p-2, 0.0, 0.0, 0.0,
};

// ---- order 11: g = 6, window 11, 14 tested candidates
template <> struct Tab<11> { static constexpr int T = 14; };
template <> struct Cand<11, 0> { static constexpr int m = 5, n = 5; };
template <> struct Cand<11, 1> { static constexpr int m = 4, n = 5; };
template <> struct Cand<11, 2> { static constexpr int m = 5, n = 4; };
template <> struct Cand<11, 3> { static constexpr int m = 4, n = 4; };
template <> struct Cand<11, 4> { static constexpr int m = 5, n = 3; };
template <> struct Cand<11, 5> { static constexpr int m = 3, n = 4; };
template <> struct Cand<11, 6> { static constexpr int m = 4, n = 3; };
template <> struct Cand<11, 7> { static constexpr int m = 3, n = 3; };
template <> struct Cand<11, 8> { static constexpr int m = 2, n = 3; };
template <> struct Cand<11, 9> { static constexpr int m = 3, n = 2; };
template <> struct Cand<11, 10> { static constexpr int m = 2, n = 2; };
template <> struct Cand<11, 11> { static constexpr int m = 1, n = 2; };
template <> struct Cand<11, 12> { static constexpr int m = 2, n = 1; };
template <> struct Cand<11, 13> { static constexpr int m = 1, n = 1; };
// b_l (rows t, columns l = -(g-1)..g-1; zero outside the stencil)
static __constant__ double kB11[154] = {
    1.0, -10.0, 45.0, -120.0, 210.0, -252.0, 210.0, -120.0, 45.0, -10.0, 1.0,
    0.0, -1.0, 9.0, -36.0, 84.0, -126.0, 126.0, -84.0, 36.0, -9.0, 1.0,
    -1.0, 9.0, -36.0, 84.0, -126.0, 126.0, -84.0, 36.0, -9.0, 1.0, 0.0,
    0.0, 1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0, 0.0,
    1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0,
    0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0, 0.0,
    0.0, 0.0, 1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 1.0, -4.0, 6.0, -4.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 1.0, -2.0, 1.0, 0.0, 0.0, 0.0, 0.0,
};
// a_l (same layout)
static __constant__ double kA11[154] = {
    -0x1.7a463005e918cp-12, 0x1.206f1e37b4efbp-8, -0x1.9f82b259b13e0p-6, 0x1.7fbdcd51322a7p-4, -0x1.0dc768196a50dp-2, 0x1.791c4bf34ad79p-1, 0x1.23c6f69df5824p-1, -0x1.27bf933f0564bp-3, 0x1.17dd20bac5dafp-5, -0x1.69b9845273b2ep-8, 0x1.c5edd33a4aea8p-12,
    0.0, 0x1.a01a01a01a01ap-11, -0x1.2b12b12b12b13p-7, 0x1.9cd9cd9cd9cdap-5, -0x1.8068068068068p-3, 0x1.4a90a90a90a91p-1, 0x1.4a90a90a90a91p-1, -0x1.8068068068068p-3, 0x1.9cd9cd9cd9cdap-5, -0x1.2b12b12b12b13p-7, 0x1.a01a01a01a01ap-11,
    -0x1.a01a01a01a01ap-11, 0x1.1e11e11e11e12p-7, -0x1.6f56f56f56f57p-5, 0x1.2a42a42a42a43p-3, -0x1.6adeadeadeadfp-2, 0x1.b0f70f70f70f7p-1, 0x1.ea76a76a76a77p-2, -0x1.7ab7ab7ab7ab8p-4, 0x1.e11e11e11e11ep-7, -0x1.3813813813814p-10, 0.0,
    0.0, 0x1.a01a01a01a01ap-10, -0x1.0a90a90a90a91p-6, 0x1.4374374374374p-4, -0x1.0478478478478p-2, 0x1.7dc3dc3dc3dc4p-1, 0x1.175d75d75d75dp-1, -0x1.efbefbefbefbfp-4, 0x1.6596596596596p-6, -0x1.0410410410410p-9, 0.0,
    -0x1.0410410410410p-9, 0x1.3e93e93e93e94p-6, -0x1.6736736736736p-4, 0x1.f70f70f70f70fp-3, -0x1.023c23c23c23cp-1, 0x1.fdc3dc3dc3dc4p-1, 0x1.8410410410410p-2, -0x1.9659659659659p-5, 0x1.0410410410410p-8, 0.0, 0.0,
    0.0, 0.0, -0x1.d41d41d41d41dp-9, 0x1.1ad1ad1ad1ad2p-5, -0x1.52e52e52e52e5p-3, 0x1.44e04e04e04e0p-1, 0x1.44e04e04e04e0p-1, -0x1.52e52e52e52e5p-3, 0x1.1ad1ad1ad1ad2p-5, -0x1.d41d41d41d41dp-9, 0.0,
    0.0, 0x1.d41d41d41d41dp-9, -0x1.0750750750750p-5, 0x1.1381381381381p-3, -0x1.763f63f63f63fp-2, 0x1.c4e04e04e04e0p-1, 0x1.bcf3cf3cf3cf4p-2, -0x1.0c30c30c30c31p-4, 0x1.8618618618618p-8, 0.0, 0.0,
    0.0, 0.0, -0x1.d41d41d41d41dp-8, 0x1.e79e79e79e79ep-5, -0x1.ec7ec7ec7ec7fp-3, 0x1.84e04e04e04e0p-1, 0x1.04e04e04e04e0p-1, -0x1.7297297297297p-4, 0x1.3813813813814p-7, 0.0, 0.0,
    0.0, 0.0, 0.0, 0x1.1111111111111p-6, -0x1.1111111111111p-3, 0x1.3bbbbbbbbbbbcp-1, 0x1.3bbbbbbbbbbbcp-1, -0x1.1111111111111p-3, 0x1.1111111111111p-6, 0.0, 0.0,
    0.0, 0.0, -0x1.1111111111111p-6, 0x1.ddddddddddddep-4, -0x1.8888888888889p-2, 0x1.e666666666666p-1, 0x1.7777777777777p-2, -0x1.1111111111111p-5, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0x1.1111111111111p-5, -0x1.bbbbbbbbbbbbcp-3, 0x1.9111111111111p-1, 0x1.ccccccccccccdp-2, -0x1.999999999999ap-5, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -0x1.5555555555555p-4, 0x1.2aaaaaaaaaaabp-1, 0x1.2aaaaaaaaaaabp-1, -0x1.5555555555555p-4, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0x1.5555555555555p-4, -0x1.aaaaaaaaaaaabp-2, 0x1.1555555555555p+0, 0x1.0000000000000p-2, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -0x1.5555555555555p-3, 0x1.aaaaaaaaaaaabp-1, 0x1.5555555555555p-2, 0.0, 0.0, 0.0, 0.0,
};

// ---- order 13: g = 7, window 13, 18 tested candidates
template <> struct Tab<13> { static constexpr int T = 18; };
template <> struct Cand<13, 0> { static constexpr int m = 6, n = 6; };
template <> struct Cand<13, 1> { static constexpr int m = 5, n = 6; };
template <> struct Cand<13, 2> { static constexpr int m = 6, n = 5; };
template <> struct Cand<13, 3> { static constexpr int m = 5, n = 5; };
template <> struct Cand<13, 4> { static constexpr int m = 6, n = 4; };
template <> struct Cand<13, 5> { static constexpr int m = 4, n = 5; };
template <> struct Cand<13, 6> { static constexpr int m = 5, n = 4; };
template <> struct Cand<13, 7> { static constexpr int m = 4, n = 4; };
template <> struct Cand<13, 8> { static constexpr int m = 5, n = 3; };
template <> struct Cand<13, 9> { static constexpr int m = 3, n = 4; };
template <> struct Cand<13, 10> { static constexpr int m = 4, n = 3; };
template <> struct Cand<13, 11> { static constexpr int m = 3, n = 3; };
template <> struct Cand<13, 12> { static constexpr int m = 2, n = 3; };
template <> struct Cand<13, 13> { static constexpr int m = 3, n = 2; };
template <> struct Cand<13, 14> { static constexpr int m = 2, n = 2; };
template <> struct Cand<13, 15> { static constexpr int m = 1, n = 2; };
template <> struct Cand<13, 16> { static constexpr int m = 2, n = 1; };
template <> struct Cand<13, 17> { static constexpr int m = 1, n = 1; };
// b_l (rows t, columns l = -(g-1)..g-1; zero outside the stencil)
static __constant__ double kB13[234] = {
    1.0, -12.0, 66.0, -220.0, 495.0, -792.0, 924.0, -792.0, 495.0, -220.0, 66.0, -12.0, 1.0,
    0.0, -1.0, 11.0, -55.0, 165.0, -330.0, 462.0, -462.0, 330.0, -165.0, 55.0, -11.0, 1.0,
    -1.0, 11.0, -55.0, 165.0, -330.0, 462.0, -462.0, 330.0, -165.0, 55.0, -11.0, 1.0, 0.0,
    0.0, 1.0, -10.0, 45.0, -120.0, 210.0, -252.0, 210.0, -120.0, 45.0, -10.0, 1.0, 0.0,
    1.0, -10.0, 45.0, -120.0, 210.0, -252.0, 210.0, -120.0, 45.0, -10.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 9.0, -36.0, 84.0, -126.0, 126.0, -84.0, 36.0, -9.0, 1.0, 0.0,
    0.0, -1.0, 9.0, -36.0, 84.0, -126.0, 126.0, -84.0, 36.0, -9.0, 1.0, 0.0, 0.0,
    0.0, 0.0, 1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0, 0.0, 0.0,
    0.0, 1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 1.0, -4.0, 6.0, -4.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 1.0, -2.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
};
// a_l (same layout)
static __constant__ double kA13[234] = {
    0x1.5d2d18a2fe8d0p-14, -0x1.352a987afc0cep-10, 0x1.033ebf8ee1a85p-7, -0x1.1485a5719ceb4p-5, 0x1.aea0bb8015189p-4, -0x1.1457d11ffab9ep-2, 0x1.75d4177002a31p-1, 0x1.2caf8526de10dp-1, -0x1.4d41eb6487bcep-3, 0x1.75a2fd188bb74p-5, -0x1.45e5d2ba42ea0p-7, 0x1.73ba245c7452fp-10, -0x1.975f4768d3a48p-14,
    0.0, -0x1.7a463005e918cp-13, 0x1.3ccdfb6b599e5p-9, -0x1.f9f1136e4e2abp-7, 0x1.05d62ed74a8bfp-4, -0x1.a1a731b8ed033p-3, 0x1.4e71a148a02cfp-1, 0x1.4e71a148a02cfp-1, -0x1.a1a731b8ed033p-3, 0x1.05d62ed74a8bfp-4, -0x1.f9f1136e4e2abp-7, 0x1.3ccdfb6b599e5p-9, -0x1.7a463005e918cp-13,
    0x1.7a463005e918cp-13, -0x1.33590704cd642p-9, 0x1.d54be060eec92p-7, -0x1.c3909620a7dbfp-5, 0x1.39c6852280b3bp-3, -0x1.631cbd6ebfa63p-2, 0x1.a3c6f69df5824p-1, 0x1.054d0eff7b9aap-1, -0x1.d5978804232afp-4, 0x1.8d3018d3018d3p-6, -0x1.cf62c7a0d724cp-9, 0x1.08cabb37565e2p-12, 0.0,
    0.0, -0x1.7a463005e918cp-12, 0x1.206f1e37b4efbp-8, -0x1.9f82b259b13e0p-6, 0x1.7fbdcd51322a7p-4, -0x1.0dc768196a50dp-2, 0x1.791c4bf34ad79p-1, 0x1.23c6f69df5824p-1, -0x1.27bf933f0564bp-3, 0x1.17dd20bac5dafp-5, -0x1.69b9845273b2ep-8, 0x1.c5edd33a4aea8p-12, 0.0,
    0x1.c5edd33a4aea8p-12, -0x1.4fb7e4387212cp-8, 0x1.ce342914059d7p-6, -0x1.8c72f5bafe98ap-4, 0x1.e4712fcd2b5e6p-3, -0x1.da9434e6371dap-2, 0x1.df82b259b13e0p-1, 0x1.b544c8a9a1dffp-2, -0x1.2aecdd5978804p-4, 0x1.5343bfdee6a8ap-7, -0x1.8d3018d3018d3p-11, 0.0, 0.0,
    0.0, 0.0, 0x1.a01a01a01a01ap-11, -0x1.2b12b12b12b13p-7, 0x1.9cd9cd9cd9cdap-5, -0x1.8068068068068p-3, 0x1.4a90a90a90a91p-1, 0x1.4a90a90a90a91p-1, -0x1.8068068068068p-3, 0x1.9cd9cd9cd9cdap-5, -0x1.2b12b12b12b13p-7, 0x1.a01a01a01a01ap-11, 0.0,
    0.0, -0x1.a01a01a01a01ap-11, 0x1.1e11e11e11e12p-7, -0x1.6f56f56f56f57p-5, 0x1.2a42a42a42a43p-3, -0x1.6adeadeadeadfp-2, 0x1.b0f70f70f70f7p-1, 0x1.ea76a76a76a77p-2, -0x1.7ab7ab7ab7ab8p-4, 0x1.e11e11e11e11ep-7, -0x1.3813813813814p-10, 0.0, 0.0,
    0.0, 0.0, 0x1.a01a01a01a01ap-10, -0x1.0a90a90a90a91p-6, 0x1.4374374374374p-4, -0x1.0478478478478p-2, 0x1.7dc3dc3dc3dc4p-1, 0x1.175d75d75d75dp-1, -0x1.efbefbefbefbfp-4, 0x1.6596596596596p-6, -0x1.0410410410410p-9, 0.0, 0.0,
    0.0, -0x1.0410410410410p-9, 0x1.3e93e93e93e94p-6, -0x1.6736736736736p-4, 0x1.f70f70f70f70fp-3, -0x1.023c23c23c23cp-1, 0x1.fdc3dc3dc3dc4p-1, 0x1.8410410410410p-2, -0x1.9659659659659p-5, 0x1.0410410410410p-8, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.d41d41d41d41dp-9, 0x1.1ad1ad1ad1ad2p-5, -0x1.52e52e52e52e5p-3, 0x1.44e04e04e04e0p-1, 0x1.44e04e04e04e0p-1, -0x1.52e52e52e52e5p-3, 0x1.1ad1ad1ad1ad2p-5, -0x1.d41d41d41d41dp-9, 0.0, 0.0,
    0.0, 0.0, 0x1.d41d41d41d41dp-9, -0x1.0750750750750p-5, 0x1.1381381381381p-3, -0x1.763f63f63f63fp-2, 0x1.c4e04e04e04e0p-1, 0x1.bcf3cf3cf3cf4p-2, -0x1.0c30c30c30c31p-4, 0x1.8618618618618p-8, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.d41d41d41d41dp-8, 0x1.e79e79e79e79ep-5, -0x1.ec7ec7ec7ec7fp-3, 0x1.84e04e04e04e0p-1, 0x1.04e04e04e04e0p-1, -0x1.7297297297297p-4, 0x1.3813813813814p-7, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0x1.1111111111111p-6, -0x1.1111111111111p-3, 0x1.3bbbbbbbbbbbcp-1, 0x1.3bbbbbbbbbbbcp-1, -0x1.1111111111111p-3, 0x1.1111111111111p-6, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.1111111111111p-6, 0x1.ddddddddddddep-4, -0x1.8888888888889p-2, 0x1.e666666666666p-1, 0x1.7777777777777p-2, -0x1.1111111111111p-5, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0x1.1111111111111p-5, -0x1.bbbbbbbbbbbbcp-3, 0x1.9111111111111p-1, 0x1.ccccccccccccdp-2, -0x1.999999999999ap-5, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -0x1.5555555555555p-4, 0x1.2aaaaaaaaaaabp-1, 0x1.2aaaaaaaaaaabp-1, -0x1.5555555555555p-4, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0x1.5555555555555p-4, -0x1.aaaaaaaaaaaabp-2, 0x1.1555555555555p+0, 0x1.0000000000000p-2, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -0x1.5555555555555p-3, 0x1.aaaaaaaaaaaabp-1, 0x1.5555555555555p-2, 0.0, 0.0, 0.0, 0.0, 0.0,
};

// ---- order 15: g = 8, window 15, 22 tested candidates
template <> struct Tab<15> { static constexpr int T = 22; };
template <> struct Cand<15, 0> { static constexpr int m = 7, n = 7; };
template <> struct Cand<15, 1> { static constexpr int m = 6, n = 7; };
template <> struct Cand<15, 2> { static constexpr int m = 7, n = 6; };
template <> struct Cand<15, 3> { static constexpr int m = 6, n = 6; };
template <> struct Cand<15, 4> { static constexpr int m = 7, n = 5; };
template <> struct Cand<15, 5> { static constexpr int m = 5, n = 6; };
template <> struct Cand<15, 6> { static constexpr int m = 6, n = 5; };
template <> struct Cand<15, 7> { static constexpr int m = 5, n = 5; };
template <> struct Cand<15, 8> { static constexpr int m = 6, n = 4; };
template <> struct Cand<15, 9> { static constexpr int m = 4, n = 5; };
template <> struct Cand<15, 10> { static constexpr int m = 5, n = 4; };
template <> struct Cand<15, 11> { static constexpr int m = 4, n = 4; };
template <> struct Cand<15, 12> { static constexpr int m = 5, n = 3; };
template <> struct Cand<15, 13> { static constexpr int m = 3, n = 4; };
template <> struct Cand<15, 14> { static constexpr int m = 4, n = 3; };
template <> struct Cand<15, 15> { static constexpr int m = 3, n = 3; };
template <> struct Cand<15, 16> { static constexpr int m = 2, n = 3; };
template <> struct Cand<15, 17> { static constexpr int m = 3, n = 2; };
template <> struct Cand<15, 18> { static constexpr int m = 2, n = 2; };
template <> struct Cand<15, 19> { static constexpr int m = 1, n = 2; };
template <> struct Cand<15, 20> { static constexpr int m = 2, n = 1; };
template <> struct Cand<15, 21> { static constexpr int m = 1, n = 1; };
// b_l (rows t, columns l = -(g-1)..g-1; zero outside the stencil)
static __constant__ double kB15[330] = {
    1.0, -14.0, 91.0, -364.0, 1001.0, -2002.0, 3003.0, -3432.0, 3003.0, -2002.0, 1001.0, -364.0, 91.0, -14.0, 1.0,
    0.0, -1.0, 13.0, -78.0, 286.0, -715.0, 1287.0, -1716.0, 1716.0, -1287.0, 715.0, -286.0, 78.0, -13.0, 1.0,
    -1.0, 13.0, -78.0, 286.0, -715.0, 1287.0, -1716.0, 1716.0, -1287.0, 715.0, -286.0, 78.0, -13.0, 1.0, 0.0,
    0.0, 1.0, -12.0, 66.0, -220.0, 495.0, -792.0, 924.0, -792.0, 495.0, -220.0, 66.0, -12.0, 1.0, 0.0,
    1.0, -12.0, 66.0, -220.0, 495.0, -792.0, 924.0, -792.0, 495.0, -220.0, 66.0, -12.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 11.0, -55.0, 165.0, -330.0, 462.0, -462.0, 330.0, -165.0, 55.0, -11.0, 1.0, 0.0,
    0.0, -1.0, 11.0, -55.0, 165.0, -330.0, 462.0, -462.0, 330.0, -165.0, 55.0, -11.0, 1.0, 0.0, 0.0,
    0.0, 0.0, 1.0, -10.0, 45.0, -120.0, 210.0, -252.0, 210.0, -120.0, 45.0, -10.0, 1.0, 0.0, 0.0,
    0.0, 1.0, -10.0, 45.0, -120.0, 210.0, -252.0, 210.0, -120.0, 45.0, -10.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 9.0, -36.0, 84.0, -126.0, 126.0, -84.0, 36.0, -9.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 9.0, -36.0, 84.0, -126.0, 126.0, -84.0, 36.0, -9.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 1.0, -4.0, 6.0, -4.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, -2.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
};
// a_l (same layout)
static __constant__ double kA15[330] = {
    -0x1.45e5d2ba42ea0p-16, 0x1.48cebb775a5e6p-12, -0x1.3b59870ccde42p-9, 0x1.808c65dda3abbp-7, -0x1.524981af60c78p-5, 0x1.d40311a5776ecp-4, -0x1.19381f24db07ep-2, 0x1.7363f06d927c1p-1, 0x1.3363f06d927c1p-1, -0x1.6b53cc82999dfp-3, 0x1.ca28456d10ffap-5, -0x1.e44cd06fefb93p-7, 0x1.7bbaa46474d2fp-9, -0x1.8018018018018p-12, 0x1.74745e8bba300p-16,
    0.0, 0x1.5d2d18a2fe8d0p-15, -0x1.4ea08cf189472p-11, 0x1.31b6041a7032ap-8, -0x1.65ff1a202da5cp-6, 0x1.34b91d062d7a2p-4, -0x1.baf8c6d23e984p-3, 0x1.5141ce4b7059fp-1, 0x1.5141ce4b7059fp-1, -0x1.baf8c6d23e984p-3, 0x1.34b91d062d7a2p-4, -0x1.65ff1a202da5cp-6, 0x1.31b6041a7032ap-8, -0x1.4ea08cf189472p-11, 0x1.5d2d18a2fe8d0p-15,
    -0x1.5d2d18a2fe8d0p-15, 0x1.475a4718cea43p-11, -0x1.2212212212212p-8, 0x1.44ab908a7d04ep-6, -0x1.042a7132b6142p-4, 0x1.4507392dc167cp-3, -0x1.5d7c63691f4c2p-2, 0x1.9a66609494ec3p-1, 0x1.1141ce4b7059fp-1, -0x1.104e1c2793edap-3, 0x1.141ce4b7059eep-5, -0x1.b7042a7132b61p-8, 0x1.cbbfa4b479d34p-11, -0x1.d191762ea8bc0p-15, 0.0,
    0.0, 0x1.5d2d18a2fe8d0p-14, -0x1.352a987afc0cep-10, 0x1.033ebf8ee1a85p-7, -0x1.1485a5719ceb4p-5, 0x1.aea0bb8015189p-4, -0x1.1457d11ffab9ep-2, 0x1.75d4177002a31p-1, 0x1.2caf8526de10dp-1, -0x1.4d41eb6487bcep-3, 0x1.75a2fd188bb74p-5, -0x1.45e5d2ba42ea0p-7, 0x1.73ba245c7452fp-10, -0x1.975f4768d3a48p-14, 0.0,
    -0x1.975f4768d3a48p-14, 0x1.60d03b8f5bde8p-10, -0x1.1ee362934079ep-7, 0x1.245de8c746a2fp-5, -0x1.a6b499d5403ccp-4, 0x1.d7505dc00a8c5p-3, -0x1.bf027bcaa5648p-2, 0x1.cb296cc557f87p-1, 0x1.d95f0a4dbc219p-2, -0x1.7e120fac9db29p-4, 0x1.24298869fafccp-6, -0x1.369f0cd987c71p-9, 0x1.45e5d2ba42ea0p-13, 0.0, 0.0,
    0.0, 0.0, -0x1.7a463005e918cp-13, 0x1.3ccdfb6b599e5p-9, -0x1.f9f1136e4e2abp-7, 0x1.05d62ed74a8bfp-4, -0x1.a1a731b8ed033p-3, 0x1.4e71a148a02cfp-1, 0x1.4e71a148a02cfp-1, -0x1.a1a731b8ed033p-3, 0x1.05d62ed74a8bfp-4, -0x1.f9f1136e4e2abp-7, 0x1.3ccdfb6b599e5p-9, -0x1.7a463005e918cp-13, 0.0,
    0.0, 0x1.7a463005e918cp-13, -0x1.33590704cd642p-9, 0x1.d54be060eec92p-7, -0x1.c3909620a7dbfp-5, 0x1.39c6852280b3bp-3, -0x1.631cbd6ebfa63p-2, 0x1.a3c6f69df5824p-1, 0x1.054d0eff7b9aap-1, -0x1.d5978804232afp-4, 0x1.8d3018d3018d3p-6, -0x1.cf62c7a0d724cp-9, 0x1.08cabb37565e2p-12, 0.0, 0.0,
    0.0, 0.0, -0x1.7a463005e918cp-12, 0x1.206f1e37b4efbp-8, -0x1.9f82b259b13e0p-6, 0x1.7fbdcd51322a7p-4, -0x1.0dc768196a50dp-2, 0x1.791c4bf34ad79p-1, 0x1.23c6f69df5824p-1, -0x1.27bf933f0564bp-3, 0x1.17dd20bac5dafp-5, -0x1.69b9845273b2ep-8, 0x1.c5edd33a4aea8p-12, 0.0, 0.0,
    0.0, 0x1.c5edd33a4aea8p-12, -0x1.4fb7e4387212cp-8, 0x1.ce342914059d7p-6, -0x1.8c72f5bafe98ap-4, 0x1.e4712fcd2b5e6p-3, -0x1.da9434e6371dap-2, 0x1.df82b259b13e0p-1, 0x1.b544c8a9a1dffp-2, -0x1.2aecdd5978804p-4, 0x1.5343bfdee6a8ap-7, -0x1.8d3018d3018d3p-11, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0x1.a01a01a01a01ap-11, -0x1.2b12b12b12b13p-7, 0x1.9cd9cd9cd9cdap-5, -0x1.8068068068068p-3, 0x1.4a90a90a90a91p-1, 0x1.4a90a90a90a91p-1, -0x1.8068068068068p-3, 0x1.9cd9cd9cd9cdap-5, -0x1.2b12b12b12b13p-7, 0x1.a01a01a01a01ap-11, 0.0, 0.0,
    0.0, 0.0, -0x1.a01a01a01a01ap-11, 0x1.1e11e11e11e12p-7, -0x1.6f56f56f56f57p-5, 0x1.2a42a42a42a43p-3, -0x1.6adeadeadeadfp-2, 0x1.b0f70f70f70f7p-1, 0x1.ea76a76a76a77p-2, -0x1.7ab7ab7ab7ab8p-4, 0x1.e11e11e11e11ep-7, -0x1.3813813813814p-10, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0x1.a01a01a01a01ap-10, -0x1.0a90a90a90a91p-6, 0x1.4374374374374p-4, -0x1.0478478478478p-2, 0x1.7dc3dc3dc3dc4p-1, 0x1.175d75d75d75dp-1, -0x1.efbefbefbefbfp-4, 0x1.6596596596596p-6, -0x1.0410410410410p-9, 0.0, 0.0, 0.0,
    0.0, 0.0, -0x1.0410410410410p-9, 0x1.3e93e93e93e94p-6, -0x1.6736736736736p-4, 0x1.f70f70f70f70fp-3, -0x1.023c23c23c23cp-1, 0x1.fdc3dc3dc3dc4p-1, 0x1.8410410410410p-2, -0x1.9659659659659p-5, 0x1.0410410410410p-8, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -0x1.d41d41d41d41dp-9, 0x1.1ad1ad1ad1ad2p-5, -0x1.52e52e52e52e5p-3, 0x1.44e04e04e04e0p-1, 0x1.44e04e04e04e0p-1, -0x1.52e52e52e52e5p-3, 0x1.1ad1ad1ad1ad2p-5, -0x1.d41d41d41d41dp-9, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0x1.d41d41d41d41dp-9, -0x1.0750750750750p-5, 0x1.1381381381381p-3, -0x1.763f63f63f63fp-2, 0x1.c4e04e04e04e0p-1, 0x1.bcf3cf3cf3cf4p-2, -0x1.0c30c30c30c31p-4, 0x1.8618618618618p-8, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -0x1.d41d41d41d41dp-8, 0x1.e79e79e79e79ep-5, -0x1.ec7ec7ec7ec7fp-3, 0x1.84e04e04e04e0p-1, 0x1.04e04e04e04e0p-1, -0x1.7297297297297p-4, 0x1.3813813813814p-7, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0x1.1111111111111p-6, -0x1.1111111111111p-3, 0x1.3bbbbbbbbbbbcp-1, 0x1.3bbbbbbbbbbbcp-1, -0x1.1111111111111p-3, 0x1.1111111111111p-6, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -0x1.1111111111111p-6, 0x1.ddddddddddddep-4, -0x1.8888888888889p-2, 0x1.e666666666666p-1, 0x1.7777777777777p-2, -0x1.1111111111111p-5, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0x1.1111111111111p-5, -0x1.bbbbbbbbbbbbcp-3, 0x1.9111111111111p-1, 0x1.ccccccccccccdp-2, -0x1.999999999999ap-5, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -0x1.5555555555555p-4, 0x1.2aaaaaaaaaaabp-1, 0x1.2aaaaaaaaaaabp-1, -0x1.5555555555555p-4, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0x1.5555555555555p-4, -0x1.aaaaaaaaaaaabp-2, 0x1.1555555555555p+0, 0x1.0000000000000p-2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -0x1.5555555555555p-3, 0x1.aaaaaaaaaaaabp-1, 0x1.5555555555555p-2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
};

// ---- order 17: g = 9, window 17, 26 tested candidates
template <> struct Tab<17> { static constexpr int T = 26; };
template <> struct Cand<17, 0> { static constexpr int m = 8, n = 8; };
template <> struct Cand<17, 1> { static constexpr int m = 7, n = 8; };
template <> struct Cand<17, 2> { static constexpr int m = 8, n = 7; };
template <> struct Cand<17, 3> { static constexpr int m = 7, n = 7; };
template <> struct Cand<17, 4> { static constexpr int m = 8, n = 6; };
template <> struct Cand<17, 5> { static constexpr int m = 6, n = 7; };
template <> struct Cand<17, 6> { static constexpr int m = 7, n = 6; };
template <> struct Cand<17, 7> { static constexpr int m = 6, n = 6; };
template <> struct Cand<17, 8> { static constexpr int m = 7, n = 5; };
template <> struct Cand<17, 9> { static constexpr int m = 5, n = 6; };
template <> struct Cand<17, 10> { static constexpr int m = 6, n = 5; };
template <> struct Cand<17, 11> { static constexpr int m = 5, n = 5; };
template <> struct Cand<17, 12> { static constexpr int m = 6, n = 4; };
template <> struct Cand<17, 13> { static constexpr int m = 4, n = 5; };
template <> struct Cand<17, 14> { static constexpr int m = 5, n = 4; };
template <> struct Cand<17, 15> { static constexpr int m = 4, n = 4; };
template <> struct Cand<17, 16> { static constexpr int m = 5, n = 3; };
template <> struct Cand<17, 17> { static constexpr int m = 3, n = 4; };
template <> struct Cand<17, 18> { static constexpr int m = 4, n = 3; };
template <> struct Cand<17, 19> { static constexpr int m = 3, n = 3; };
template <> struct Cand<17, 20> { static constexpr int m = 2, n = 3; };
template <> struct Cand<17, 21> { static constexpr int m = 3, n = 2; };
template <> struct Cand<17, 22> { static constexpr int m = 2, n = 2; };
template <> struct Cand<17, 23> { static constexpr int m = 1, n = 2; };
template <> struct Cand<17, 24> { static constexpr int m = 2, n = 1; };
template <> struct Cand<17, 25> { static constexpr int m = 1, n = 1; };
// b_l (rows t, columns l = -(g-1)..g-1; zero outside the stencil)
static __constant__ double kB17[442] = {
    1.0, -16.0, 120.0, -560.0, 1820.0, -4368.0, 8008.0, -11440.0, 12870.0, -11440.0, 8008.0, -4368.0, 1820.0, -560.0, 120.0, -16.0, 1.0,
    0.0, -1.0, 15.0, -105.0, 455.0, -1365.0, 3003.0, -5005.0, 6435.0, -6435.0, 5005.0, -3003.0, 1365.0, -455.0, 105.0, -15.0, 1.0,
    -1.0, 15.0, -105.0, 455.0, -1365.0, 3003.0, -5005.0, 6435.0, -6435.0, 5005.0, -3003.0, 1365.0, -455.0, 105.0, -15.0, 1.0, 0.0,
    0.0, 1.0, -14.0, 91.0, -364.0, 1001.0, -2002.0, 3003.0, -3432.0, 3003.0, -2002.0, 1001.0, -364.0, 91.0, -14.0, 1.0, 0.0,
    1.0, -14.0, 91.0, -364.0, 1001.0, -2002.0, 3003.0, -3432.0, 3003.0, -2002.0, 1001.0, -364.0, 91.0, -14.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 13.0, -78.0, 286.0, -715.0, 1287.0, -1716.0, 1716.0, -1287.0, 715.0, -286.0, 78.0, -13.0, 1.0, 0.0,
    0.0, -1.0, 13.0, -78.0, 286.0, -715.0, 1287.0, -1716.0, 1716.0, -1287.0, 715.0, -286.0, 78.0, -13.0, 1.0, 0.0, 0.0,
    0.0, 0.0, 1.0, -12.0, 66.0, -220.0, 495.0, -792.0, 924.0, -792.0, 495.0, -220.0, 66.0, -12.0, 1.0, 0.0, 0.0,
    0.0, 1.0, -12.0, 66.0, -220.0, 495.0, -792.0, 924.0, -792.0, 495.0, -220.0, 66.0, -12.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 11.0, -55.0, 165.0, -330.0, 462.0, -462.0, 330.0, -165.0, 55.0, -11.0, 1.0, 0.0, 0.0,
    0.0, 0.0, -1.0, 11.0, -55.0, 165.0, -330.0, 462.0, -462.0, 330.0, -165.0, 55.0, -11.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 1.0, -10.0, 45.0, -120.0, 210.0, -252.0, 210.0, -120.0, 45.0, -10.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 1.0, -10.0, 45.0, -120.0, 210.0, -252.0, 210.0, -120.0, 45.0, -10.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -1.0, 9.0, -36.0, 84.0, -126.0, 126.0, -84.0, 36.0, -9.0, 1.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -1.0, 9.0, -36.0, 84.0, -126.0, 126.0, -84.0, 36.0, -9.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 1.0, -8.0, 28.0, -56.0, 70.0, -56.0, 28.0, -8.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, -1.0, 7.0, -21.0, 35.0, -35.0, 21.0, -7.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 5.0, -10.0, 10.0, -5.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, -4.0, 6.0, -4.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 3.0, -3.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, -2.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
};
// a_l (same layout)
static __constant__ double kA17[442] = {
    0x1.32ba2fbe5d188p-18, -0x1.5b76ea15a575cp-14, 0x1.77940d1a7cc75p-11, -0x1.0294f3eb4f227p-8, 0x1.0028fe748615cp-6, -0x1.893aa15aaefe7p-5, 0x1.f276dac3eb37ep-4, -0x1.1cfbe2e89ecbap-2, 0x1.71820e8bb09a3p-1, 0x1.389e8052cd0bfp-1, -0x1.83ec651b32369p-3, 0x1.0ac576f37fa58p-4, -0x1.43127b1486d83p-6, 0x1.37bd3cdaa5f71p-8, -0x1.b72a81b72a81bp-11, 0x1.8d71d301ceea4p-14, -0x1.591175b628bb8p-18,
    0.0, -0x1.45e5d2ba42ea0p-17, 0x1.6016016016016p-13, -0x1.6b5c873cd0e45p-10, 0x1.df7b0ef6c0e07p-8, -0x1.cb5cb5cb5cb5dp-6, 0x1.5c8b9a2dfff74p-4, -0x1.cee2056627d6ep-3, 0x1.5363f06d927c1p-1, 0x1.5363f06d927c1p-1, -0x1.cee2056627d6ep-3, 0x1.5c8b9a2dfff74p-4, -0x1.cb5cb5cb5cb5dp-6, 0x1.df7b0ef6c0e07p-8, -0x1.6b5c873cd0e45p-10, 0x1.6016016016016p-13, -0x1.45e5d2ba42ea0p-17,
    0x1.45e5d2ba42ea0p-17, -0x1.5a442fe5e718ap-13, 0x1.5d8a35baa17b9p-10, -0x1.bf4a804aed690p-8, 0x1.997c808236af1p-6, -0x1.209c384f27db3p-4, 0x1.4d8fc1b649f04p-3, -0x1.59381f24db07ep-2, 0x1.9363f06d927c1p-1, 0x1.1a806234aeeddp-1, -0x1.2f9810c6dde24p-3, 0x1.5d8d1ea35e930p-5, -0x1.537df20dac7dbp-7, 0x1.ec1ec1ec1ec1fp-10, -0x1.cea88d719147ap-13, 0x1.a302ea5d31760p-17, 0.0,
    0.0, -0x1.45e5d2ba42ea0p-16, 0x1.48cebb775a5e6p-12, -0x1.3b59870ccde42p-9, 0x1.808c65dda3abbp-7, -0x1.524981af60c78p-5, 0x1.d40311a5776ecp-4, -0x1.19381f24db07ep-2, 0x1.7363f06d927c1p-1, 0x1.3363f06d927c1p-1, -0x1.6b53cc82999dfp-3, 0x1.ca28456d10ffap-5, -0x1.e44cd06fefb93p-7, 0x1.7bbaa46474d2fp-9, -0x1.8018018018018p-12, 0x1.74745e8bba300p-16, 0.0,
    0x1.74745e8bba300p-16, -0x1.718b75cea2bbap-12, 0x1.5aa14cfd8a073p-9, -0x1.99d3cbc85f6ebp-7, 0x1.586128fb49e33p-5, -0x1.ba35d1e8c174dp-4, 0x1.cd8fc1b649f04p-3, -0x1.ab8143b7242c7p-2, 0x1.bc8882b6b70e6p-1, 0x1.f500c4695ddbbp-2, -0x1.c59687f4222aep-4, 0x1.a3d46bd2600ecp-6, -0x1.329eccd587870p-8, 0x1.28ccbb57585e4p-11, -0x1.175746e8cba40p-15, 0.0, 0.0,
    0.0, 0.0, 0x1.5d2d18a2fe8d0p-15, -0x1.4ea08cf189472p-11, 0x1.31b6041a7032ap-8, -0x1.65ff1a202da5cp-6, 0x1.34b91d062d7a2p-4, -0x1.baf8c6d23e984p-3, 0x1.5141ce4b7059fp-1, 0x1.5141ce4b7059fp-1, -0x1.baf8c6d23e984p-3, 0x1.34b91d062d7a2p-4, -0x1.65ff1a202da5cp-6, 0x1.31b6041a7032ap-8, -0x1.4ea08cf189472p-11, 0x1.5d2d18a2fe8d0p-15, 0.0,
    0.0, -0x1.5d2d18a2fe8d0p-15, 0x1.475a4718cea43p-11, -0x1.2212212212212p-8, 0x1.44ab908a7d04ep-6, -0x1.042a7132b6142p-4, 0x1.4507392dc167cp-3, -0x1.5d7c63691f4c2p-2, 0x1.9a66609494ec3p-1, 0x1.1141ce4b7059fp-1, -0x1.104e1c2793edap-3, 0x1.141ce4b7059eep-5, -0x1.b7042a7132b61p-8, 0x1.cbbfa4b479d34p-11, -0x1.d191762ea8bc0p-15, 0.0, 0.0,
    0.0, 0.0, 0x1.5d2d18a2fe8d0p-14, -0x1.352a987afc0cep-10, 0x1.033ebf8ee1a85p-7, -0x1.1485a5719ceb4p-5, 0x1.aea0bb8015189p-4, -0x1.1457d11ffab9ep-2, 0x1.75d4177002a31p-1, 0x1.2caf8526de10dp-1, -0x1.4d41eb6487bcep-3, 0x1.75a2fd188bb74p-5, -0x1.45e5d2ba42ea0p-7, 0x1.73ba245c7452fp-10, -0x1.975f4768d3a48p-14, 0.0, 0.0,
    0.0, -0x1.975f4768d3a48p-14, 0x1.60d03b8f5bde8p-10, -0x1.1ee362934079ep-7, 0x1.245de8c746a2fp-5, -0x1.a6b499d5403ccp-4, 0x1.d7505dc00a8c5p-3, -0x1.bf027bcaa5648p-2, 0x1.cb296cc557f87p-1, 0x1.d95f0a4dbc219p-2, -0x1.7e120fac9db29p-4, 0x1.24298869fafccp-6, -0x1.369f0cd987c71p-9, 0x1.45e5d2ba42ea0p-13, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.7a463005e918cp-13, 0x1.3ccdfb6b599e5p-9, -0x1.f9f1136e4e2abp-7, 0x1.05d62ed74a8bfp-4, -0x1.a1a731b8ed033p-3, 0x1.4e71a148a02cfp-1, 0x1.4e71a148a02cfp-1, -0x1.a1a731b8ed033p-3, 0x1.05d62ed74a8bfp-4, -0x1.f9f1136e4e2abp-7, 0x1.3ccdfb6b599e5p-9, -0x1.7a463005e918cp-13, 0.0, 0.0,
    0.0, 0.0, 0x1.7a463005e918cp-13, -0x1.33590704cd642p-9, 0x1.d54be060eec92p-7, -0x1.c3909620a7dbfp-5, 0x1.39c6852280b3bp-3, -0x1.631cbd6ebfa63p-2, 0x1.a3c6f69df5824p-1, 0x1.054d0eff7b9aap-1, -0x1.d5978804232afp-4, 0x1.8d3018d3018d3p-6, -0x1.cf62c7a0d724cp-9, 0x1.08cabb37565e2p-12, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.7a463005e918cp-12, 0x1.206f1e37b4efbp-8, -0x1.9f82b259b13e0p-6, 0x1.7fbdcd51322a7p-4, -0x1.0dc768196a50dp-2, 0x1.791c4bf34ad79p-1, 0x1.23c6f69df5824p-1, -0x1.27bf933f0564bp-3, 0x1.17dd20bac5dafp-5, -0x1.69b9845273b2ep-8, 0x1.c5edd33a4aea8p-12, 0.0, 0.0, 0.0,
    0.0, 0.0, 0x1.c5edd33a4aea8p-12, -0x1.4fb7e4387212cp-8, 0x1.ce342914059d7p-6, -0x1.8c72f5bafe98ap-4, 0x1.e4712fcd2b5e6p-3, -0x1.da9434e6371dap-2, 0x1.df82b259b13e0p-1, 0x1.b544c8a9a1dffp-2, -0x1.2aecdd5978804p-4, 0x1.5343bfdee6a8ap-7, -0x1.8d3018d3018d3p-11, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0x1.a01a01a01a01ap-11, -0x1.2b12b12b12b13p-7, 0x1.9cd9cd9cd9cdap-5, -0x1.8068068068068p-3, 0x1.4a90a90a90a91p-1, 0x1.4a90a90a90a91p-1, -0x1.8068068068068p-3, 0x1.9cd9cd9cd9cdap-5, -0x1.2b12b12b12b13p-7, 0x1.a01a01a01a01ap-11, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.a01a01a01a01ap-11, 0x1.1e11e11e11e12p-7, -0x1.6f56f56f56f57p-5, 0x1.2a42a42a42a43p-3, -0x1.6adeadeadeadfp-2, 0x1.b0f70f70f70f7p-1, 0x1.ea76a76a76a77p-2, -0x1.7ab7ab7ab7ab8p-4, 0x1.e11e11e11e11ep-7, -0x1.3813813813814p-10, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0x1.a01a01a01a01ap-10, -0x1.0a90a90a90a91p-6, 0x1.4374374374374p-4, -0x1.0478478478478p-2, 0x1.7dc3dc3dc3dc4p-1, 0x1.175d75d75d75dp-1, -0x1.efbefbefbefbfp-4, 0x1.6596596596596p-6, -0x1.0410410410410p-9, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, -0x1.0410410410410p-9, 0x1.3e93e93e93e94p-6, -0x1.6736736736736p-4, 0x1.f70f70f70f70fp-3, -0x1.023c23c23c23cp-1, 0x1.fdc3dc3dc3dc4p-1, 0x1.8410410410410p-2, -0x1.9659659659659p-5, 0x1.0410410410410p-8, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -0x1.d41d41d41d41dp-9, 0x1.1ad1ad1ad1ad2p-5, -0x1.52e52e52e52e5p-3, 0x1.44e04e04e04e0p-1, 0x1.44e04e04e04e0p-1, -0x1.52e52e52e52e5p-3, 0x1.1ad1ad1ad1ad2p-5, -0x1.d41d41d41d41dp-9, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0x1.d41d41d41d41dp-9, -0x1.0750750750750p-5, 0x1.1381381381381p-3, -0x1.763f63f63f63fp-2, 0x1.c4e04e04e04e0p-1, 0x1.bcf3cf3cf3cf4p-2, -0x1.0c30c30c30c31p-4, 0x1.8618618618618p-8, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -0x1.d41d41d41d41dp-8, 0x1.e79e79e79e79ep-5, -0x1.ec7ec7ec7ec7fp-3, 0x1.84e04e04e04e0p-1, 0x1.04e04e04e04e0p-1, -0x1.7297297297297p-4, 0x1.3813813813814p-7, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.1111111111111p-6, -0x1.1111111111111p-3, 0x1.3bbbbbbbbbbbcp-1, 0x1.3bbbbbbbbbbbcp-1, -0x1.1111111111111p-3, 0x1.1111111111111p-6, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, -0x1.1111111111111p-6, 0x1.ddddddddddddep-4, -0x1.8888888888889p-2, 0x1.e666666666666p-1, 0x1.7777777777777p-2, -0x1.1111111111111p-5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.1111111111111p-5, -0x1.bbbbbbbbbbbbcp-3, 0x1.9111111111111p-1, 0x1.ccccccccccccdp-2, -0x1.999999999999ap-5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -0x1.5555555555555p-4, 0x1.2aaaaaaaaaaabp-1, 0x1.2aaaaaaaaaaabp-1, -0x1.5555555555555p-4, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.5555555555555p-4, -0x1.aaaaaaaaaaaabp-2, 0x1.1555555555555p+0, 0x1.0000000000000p-2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -0x1.5555555555555p-3, 0x1.aaaaaaaaaaaabp-1, 0x1.5555555555555p-2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
};

template <int R> struct Coef;
template <> struct Coef<5> {
    __device__ static __forceinline__ double b(int i) { return kB5[i]; }
    __device__ static __forceinline__ double a(int i) { return kA5[i]; }
    __device__ static __forceinline__ const double *a_table() { return kA5; }
};
template <> struct Coef<7> {
    __device__ static __forceinline__ double b(int i) { return kB7[i]; }
    __device__ static __forceinline__ double a(int i) { return kA7[i]; }
    __device__ static __forceinline__ const double *a_table() { return kA7; }
};
template <> struct Coef<9> {
    __device__ static __forceinline__ double b(int i) { return kB9[i]; }
    __device__ static __forceinline__ double a(int i) { return kA9[i]; }
    __device__ static __forceinline__ const double *a_table() { return kA9; }
};
template <> struct Coef<11> {
    __device__ static __forceinline__ double b(int i) { return kB11[i]; }
    __device__ static __forceinline__ double a(int i) { return kA11[i]; }
    __device__ static __forceinline__ const double *a_table() { return kA11; }
};
template <> struct Coef<13> {
    __device__ static __forceinline__ double b(int i) { return kB13[i]; }
    __device__ static __forceinline__ double a(int i) { return kA13[i]; }
    __device__ static __forceinline__ const double *a_table() { return kA13; }
};
template <> struct Coef<15> {
    __device__ static __forceinline__ double b(int i) { return kB15[i]; }
    __device__ static __forceinline__ double a(int i) { return kA15[i]; }
    __device__ static __forceinline__ const double *a_table() { return kA15; }
};
template <> struct Coef<17> {
    __device__ static __forceinline__ double b(int i) { return kB17[i]; }
    __device__ static __forceinline__ double a(int i) { return kA17[i]; }
    __device__ static __forceinline__ const double *a_table() { return kA17; }
};

}  // namespace enomr
